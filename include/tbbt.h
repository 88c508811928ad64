/*
 * tbbt -- tridiagonal -> band eigenvector back-transformation on GB300.
 *
 * C ABI of the library libtbbt.so. It computes step Eq. 6d of the two-stage
 * symmetric / Hermitian eigensolver of arXiv 2002.10991 (ELPA2),
 *
 *     Z = Q^* X = H_0 H_1 ... H_{K-1} X,      H_k = I - tau_k v_k v_k^H,
 *
 * i.e. every Householder reflector generated by the band -> tridiagonal
 * bulge chase (Eq. 6b, Eq. 7, Sec. 2.2.1) applied to an n x nev block of
 * eigenvectors in the reverse of generation order (Sec. 2.2.2), each one as
 * x <- x - tau v (v^H x) (Eq. 8). Real symmetric problems use double,
 * Hermitian problems complex double (two doubles, real part first, the
 * layout of C99 double complex, cuDoubleComplex and numpy complex128).
 *
 * ---------------------------------------------------------------------------
 * The reflector store (canonical input format)
 * ---------------------------------------------------------------------------
 * Reflectors are numbered k = 0..K-1 in generation order: stage i = 0..n-3,
 * and within stage i the sweeps j = 0..ceil((n-i-2)/b)-1 (Sec. 2.2.1; the
 * printed sweep count "(N-i)/b" is read as ceil((N-i-1)/b) with 1-based i,
 * which reproduces the paper's N=17, b=4 example). A Hermitian store ends
 * with one more reflector (stage n-2, sweep 0) of length 1 that makes the
 * last sub-diagonal entry real. Reflector k acts on rows
 *     r_k = i + 1 + j*b  ..  r_k + L_k - 1,    L_k = min(b, n - r_k)
 * (0-based rows), so r_k and L_k follow from (n, b) and need no index array.
 *
 *   hh_v    K x b, column-major: reflector k is hh_v[k*b .. k*b + b); its
 *           first entry v_k[0] = 1 is stored explicitly; entries at
 *           positions >= L_k are ignored (conventionally zero).
 *   hh_tau  K scalars tau_k (complex for Hermitian problems, LAPACK
 *           convention: H_k^H x = beta e_1 with real beta in the reduction).
 *
 * tbbt_num_reflectors(n, b, is_complex) returns K.
 *
 * ---------------------------------------------------------------------------
 * Conventions of every call
 * ---------------------------------------------------------------------------
 * - Pointers named d_* or documented as device pointers are device memory
 *   owned by the caller; the library never frees them.
 * - q is n x nev, column-major, leading dimension ldq >= max(1, n), and is
 *   overwritten with Z. Rows n..ldq-1 are never read or written.
 * - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *   stream) with no host synchronisation, except where a call says it
 *   allocates. Errors found on the host are returned at once; faults of
 *   enqueued work surface in later CUDA calls; bounded waits inside kernels
 *   that give up record TBBT_ETIMEOUT in a device word that
 *   tbbt_stream_check() reports.
 * - No exception crosses the ABI. NaN or Inf in the inputs propagates to the
 *   affected columns; it is not checked.
 * - Device: compute capability 10.3 (GB300, sm_103a).
 */
#ifndef TBBT_H
#define TBBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TBBT_OK = 0,
  TBBT_EINVAL = 1,   /* invalid argument (size, pointer, alignment, leading dimension) */
  TBBT_ENOMEM = 2,   /* device or host allocation failed */
  TBBT_ECUDA = 3,    /* a CUDA runtime call failed */
  TBBT_ETIMEOUT = 4, /* a bounded in-kernel wait gave up (reported by tbbt_stream_check) */
  TBBT_ENOTSUP = 5   /* valid request this build does not support (e.g. variant / size) */
} tbbt_status;

typedef enum { TBBT_REAL64 = 0, TBBT_COMPLEX128 = 1 } tbbt_dtype;

/* Human-readable name of a status code (static string). */
const char *tbbt_status_string(tbbt_status s);

/* Number of reflectors K in the store of an n x n problem with semi-bandwidth
 * b (Sec. 2.2.1: N-2 stages, ceil((N-i-1)/b) sweeps in 1-based stage i; one
 * more for Hermitian problems). Returns -1 for n < 0 or b < 1. */
int64_t tbbt_num_reflectors(int64_t n, int64_t b, int is_complex);

/* ---------------------------------------------------------------------------
 * One-shot calls (Eq. 6d). hh_v, hh_tau and q are device pointers.
 *
 * n >= 0, 1 <= nbw <= 128, 0 <= nev <= n, ldq >= max(1, n); q aligned to its
 * element size. The first call for a given (dtype, n, nbw, nev) allocates a
 * cached workspace (a host-synchronising cudaMalloc); later calls with the
 * same shape reuse it and do not synchronise. Calls sharing a shape must not
 * overlap on different streams (they share the workspace); use plans for
 * that. The cache lives until tbbt_release_cache() or process exit.
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_trans_ev_tridi_to_band_d(const double *hh_v, const double *hh_tau, int64_t n, int64_t nbw,
                                          int64_t nev, double *q, int64_t ldq, void *stream);
/* Complex double: each pointer addresses interleaved (re, im) pairs. */
tbbt_status tbbt_trans_ev_tridi_to_band_z(const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw,
                                          int64_t nev, void *q, int64_t ldq, void *stream);

/* Same computation with every array in HOST memory (pinned memory makes the
 * copies asynchronous). The call copies the store and X to the device, runs
 * the back-transform and copies Z back into q, all on `stream`; the caller
 * synchronises the stream before reading q. Uses the one-shot cache plus a
 * cached device copy of the inputs. */
tbbt_status tbbt_trans_ev_tridi_to_band_host_d(const double *hh_v, const double *hh_tau, int64_t n,
                                               int64_t nbw, int64_t nev, double *q, int64_t ldq, void *stream);
tbbt_status tbbt_trans_ev_tridi_to_band_host_z(const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw,
                                               int64_t nev, void *q, int64_t ldq, void *stream);

/* Frees every workspace cached by the one-shot calls (synchronises the device). */
tbbt_status tbbt_release_cache(void);

/* ---------------------------------------------------------------------------
 * Plans: all device allocation happens in tbbt_plan_create (the paper's
 * advice to pre-compute and pre-allocate workspace outside the work loop,
 * Sec. 3.1); set_reflectors and execute only enqueue kernels.
 * ------------------------------------------------------------------------- */
typedef struct tbbt_plan tbbt_plan;

typedef struct {
  /* Sweeps processed concurrently by one thread block (one warp each, two
   * for complex data); 0 = choose automatically (4 real, 1 complex). */
  int32_t sweeps_per_block;
  /* Stages each warp applies between two block-wide synchronisations;
   * 0 = choose automatically (8 real, 2 complex; at most 4 * sweeps_per_block). */
  int32_t stages_per_step;
  /* Limit of every in-kernel wait, in milliseconds; 0 = 20000. A wait that
   * runs out records TBBT_ETIMEOUT (see tbbt_stream_check); the kernel then
   * abandons the dependent work and exits. */
  int32_t wait_timeout_ms;
  /* Test hook; 0 = off. Otherwise 1 + the index of a work unit (32-column
   * strip, group of sweeps) whose progress is never published, so that the
   * units waiting for it run into wait_timeout_ms. */
  int32_t debug_withhold_unit_plus1;
  /* TBBT_VARIANT_FP64 (0, default): reflector-by-reflector FP64 arithmetic.
   * TBBT_VARIANT_SPLIT_BF16 (1): real data with nbw = 32 or 64 only. Blocks of
   * 32 consecutive reflectors of a sweep are put in compact WY form
   * (I - V T V^T, T computed in FP64 per plan by the forward recurrence) and
   * applied as two products on BF16 tensor cores, with the eigenvector block
   * held in 64-bit fixed point per column and split into 6 exact 8-bit digit
   * slices (Ozaki-style; every partial sum is exact in FP32). Error relative
   * to each column's norm ~1e-14 per block application (see the benchmark's
   * accuracy figures). Other shapes return TBBT_ENOTSUP.
   * TBBT_VARIANT_SPLIT_BF16_TC (2): the same split-precision method on the
   * fifth-generation tensor cores (tcgen05 MMA, accumulators in tensor
   * memory, operands staged by the bulk-copy engine): one thread block per SM
   * owning 128-column strips, the eigenvector window held in registers.
   * Real data with nbw = 32 or 64 on an sm_100-family device; otherwise
   * TBBT_ENOTSUP. The plan also holds a 64-bit fixed-point copy of the
   * eigenvector block (nev * (n + 2) * 8 bytes). */
  int32_t variant;
  int32_t reserved[3];
} tbbt_options;

#define TBBT_VARIANT_FP64 0
#define TBBT_VARIANT_SPLIT_BF16 1
#define TBBT_VARIANT_SPLIT_BF16_TC 2

/* Creates a plan for problems of the given type and shape (arguments as for
 * the one-shot calls). opt may be NULL. Allocates the re-laid reflector
 * store (K * round_up(nbw, 2) elements) and small tables; synchronises. */
tbbt_status tbbt_plan_create(tbbt_plan **plan, tbbt_dtype dtype, int64_t n, int64_t nbw, int64_t nev,
                             const tbbt_options *opt);

/* Re-lays the canonical store (device pointers hh_v, hh_tau in the format
 * above) into the plan's sweep-major layout (Sec. 3.2: one process applies
 * consecutive reflectors of a sweep, each shifted up by one row). Enqueued on
 * `stream`; the input arrays may be reused once the stream reaches this point. */
tbbt_status tbbt_plan_set_reflectors(tbbt_plan *plan, const void *hh_v, const void *hh_tau, void *stream);

/* Applies the reflectors set last to q (device pointer, n x nev, ldq) in place. */
tbbt_status tbbt_plan_execute(tbbt_plan *plan, void *q, int64_t ldq, void *stream);

/* Destroys a plan (synchronises the device). Accepts NULL. */
tbbt_status tbbt_plan_destroy(tbbt_plan *plan);

/* Launch geometry a plan chose (for the benchmark and tests): sweeps per
 * block, stages per step, ring rows, dynamic shared memory bytes, blocks. */
tbbt_status tbbt_plan_info(const tbbt_plan *plan, int32_t *sweeps_per_block, int32_t *stages_per_step,
                           int32_t *ring_rows, int32_t *smem_bytes, int32_t *blocks);

/* ---------------------------------------------------------------------------
 * Batched form: many independent problems of uneven size (for example the
 * k-points and spin channels of one KS-DFT iteration, Sec. 5), real and
 * complex mixed, back-transformed by ONE persistent kernel launch. All
 * pointers are device pointers fixed at creation: the batch captures a CUDA
 * graph (re-layout of every store, queue reset, the persistent launch), and
 * each execute replays it on the caller's stream, reading the stores and
 * updating every q in place. Update the contents of the arrays between
 * executes, not their addresses.
 * ------------------------------------------------------------------------- */
typedef struct {
  tbbt_dtype dtype;  /* TBBT_REAL64 or TBBT_COMPLEX128 */
  int32_t reserved0;
  int64_t n, nbw, nev; /* as for the one-shot calls */
  const void *hh_v;    /* canonical store, device */
  const void *hh_tau;
  void *q; /* n x nev, column-major, device, updated in place */
  int64_t ldq;
} tbbt_problem;

typedef struct tbbt_batch tbbt_batch;

typedef struct {
  int32_t sweeps_per_block;        /* 0 = 4 (4 or 8) */
  int32_t stages_per_step_real;    /* 0 = 16 */
  int32_t stages_per_step_complex; /* 0 = 4; defaults are lowered until two blocks fit an SM */
  /* Nonzero: time candidate geometries at creation and keep the fastest.
   * Candidates run on a proxy of the batch (every problem with 1/16 of its
   * columns, in whole 32-column strips, on scratch copies; the caller's data
   * are not touched): six candidates cost about 3/4 of one execution of
   * the batch. Results are cached per process and GPU and, if
   * autotune_cache (or the environment variable TBBT_AUTOTUNE_CACHE) names
   * a file, appended to it and read back by later processes. */
  int32_t autotune;
  const char *autotune_cache;
  int32_t wait_timeout_ms; /* 0 = 20000, see tbbt_options */
  int32_t reserved[5];
} tbbt_batch_options;

/* Creates a batch of `count` problems (opt may be NULL). Allocates all
 * workspace and instantiates the graph; synchronises. */
tbbt_status tbbt_batch_create(tbbt_batch **batch, int32_t count, const tbbt_problem *problems,
                              const tbbt_batch_options *opt);
/* Enqueues one replay of the batch's graph on `stream`. */
tbbt_status tbbt_batch_execute(tbbt_batch *batch, void *stream);
/* Geometry in use: sweeps per block, stages per step (real / complex),
 * persistent blocks, queued work units, whether it came from tuning. */
tbbt_status tbbt_batch_info(const tbbt_batch *batch, int32_t *sweeps_per_block, int32_t *stages_real,
                            int32_t *stages_complex, int32_t *blocks, int64_t *units, int32_t *tuned);
/* Destroys a batch (synchronises the device). Accepts NULL. */
tbbt_status tbbt_batch_destroy(tbbt_batch *batch);

/* Synchronises `stream`, then reports (and clears) the device error word:
 * TBBT_OK, TBBT_ETIMEOUT, or TBBT_ECUDA if the stream itself failed. The
 * word is sticky: after a timeout, later launches return at once without
 * computing until this call has cleared it. */
tbbt_status tbbt_stream_check(void *stream);

/* ---------------------------------------------------------------------------
 * The same computation without any allocation (the paper has no counterpart;
 * this is a service of the library). For callers that cannot allocate device
 * memory when they call: all of the GPU may already belong to another
 * allocator, the call may sit in a loop where the host-device
 * synchronisation of cudaMalloc/cudaFree is not acceptable, or the caller
 * must not meet out-of-memory at run time.
 *
 * dtype selects real (double) or Hermitian (interleaved complex double)
 * data; the other arguments are as for tbbt_trans_ev_tridi_to_band_d/_z
 * (device pointers, q overwritten in place). Nothing is allocated: the
 * scratch (sweep-major copy of the store, stage offsets, progress flags) lives
 * in one array of TBBT_NOALLOC_SCRATCH_BYTES in the library's device code,
 * which every GPU that loads the library holds until the process exits.
 * Problems whose scratch does not fit -- about K * round_up(nbw, 2) elements
 * of 8 (real) or 16 (complex) bytes plus small tables, i.e. up to n ~ 2800
 * real or ~ 2000 complex at nbw = 64 -- return TBBT_ENOTSUP before any work.
 *
 * The first call on each device sets that device up (looks up the array's
 * device address, sets a kernel attribute); make that first call before any
 * stream capture. Every call shares the one array and leaves its contents
 * behind (the parts that must start cleared are cleared by each call), so
 * calls that overlap on the GPU -- on different streams or from different
 * host threads -- race and corrupt each other's results: serialise them.
 * ------------------------------------------------------------------------- */
#define TBBT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
tbbt_status tbbt_trans_ev_tridi_to_band_noalloc(tbbt_dtype dtype, const void *hh_v, const void *hh_tau, int64_t n,
                                                int64_t nbw, int64_t nev, void *q, int64_t ldq, void *stream);

/* -------------------------------------------------------------------------
 * Band -> tridiagonal reduction by bulge chasing (Eq. 6b, Sec. 2.2.1,
 * Fig. 2), the step whose reflectors the back-transformation applies: stage
 * i = 0 .. n-3 has ceil((n-i-2)/nbw) sweeps, sweep j builds the Householder
 * reflector of rows r = i+1+j*nbw .. r+L-1 (L = min(nbw, n-r); LAPACK
 * convention H^H x = beta e_1, H = I - tau v v^H, v[0] = 1) that annihilates
 * column i (j = 0) or the first column of the previous sweep's bulge, and
 * applies it two-sided. Hermitian input gets one more stage, n-2, whose
 * length-1 reflector makes the last sub-diagonal entry real, so d and e are
 * real. The reflectors come out in the canonical store of the
 * back-transformation calls, in generation order (stage-major), so the output
 * can go straight to tbbt_trans_ev_tridi_to_band_d/_z or a plan.
 *
 * band:  device, lower band storage of the input, (nbw+1) x n column-major:
 *        band[d + c*ldb] = B(c+d, c), d = 0 .. nbw (ldb >= nbw+1); entries
 *        outside the matrix are ignored; the diagonal's imaginary part is
 *        ignored. Not modified.
 * hh_v, hh_tau: device outputs, K x nbw (column-major, reflector k at
 *        hh_v[k*nbw ..], zeros beyond its length) and K, K = tbbt_num_reflectors.
 * d, e:  device outputs, n and n-1 doubles (diagonal, sub-diagonal of T).
 * The reduction runs in FP64 on the stream; a working copy of the band
 * ((2 nbw + 1) x n elements) and small tables are allocated stream-ordered
 * and released by the call. Errors: TBBT_EINVAL (shape, ldb, null pointer
 * with n > 0), TBBT_ENOTSUP (nbw too wide for the shared-memory block:
 * nbw > 117 complex), TBBT_ECUDA; bounded in-kernel waits record
 * TBBT_ETIMEOUT (see tbbt_stream_check).
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_bulge_chase_d(const double *band, int64_t ldb, int64_t n, int64_t nbw, double *hh_v, double *hh_tau,
                               double *d, double *e, void *stream);
tbbt_status tbbt_bulge_chase_z(const void *band, int64_t ldb, int64_t n, int64_t nbw, void *hh_v, void *hh_tau,
                               double *d, double *e, void *stream);

/* -------------------------------------------------------------------------
 * Tridiagonal eigensolver for the nev lowest eigenpairs (Eq. 6c; Sec. 2.1:
 * only the wanted eigenvectors of the tridiagonal matrix are computed), the
 * step whose eigenvectors X the back-transformation Eq. 6d takes. T is the
 * real symmetric tridiagonal matrix with diagonal d[0..n-1] and
 * sub-diagonal e[0..n-2] (the d, e of tbbt_bulge_chase_*).
 *
 * Eigenvalues by multisection on Sturm counts, eigenvectors by inverse
 * iteration with a pivoted tridiagonal LU (three solves from a
 * pseudo-random start), then modified Gram-Schmidt inside every cluster of
 * eigenvalues chained by gaps below 1e-4 ||T||. All in FP64.
 *
 * d, e:  device, n and n-1 doubles; read only.
 * w:     device output, nev doubles: the nev smallest eigenvalues, ascending.
 * x:     device output, n x nev column-major, ldx >= max(1, n): the
 *        orthonormal eigenvectors (column k belongs to w[k]; its entry of
 *        largest magnitude is positive, unless re-orthogonalisation in a
 *        cluster changed it). xtype TBBT_REAL64: doubles; TBBT_COMPLEX128:
 *        interleaved complex doubles with zero imaginary parts (the X of a
 *        Hermitian problem). Rows n..ldx-1 are not written.
 * Runs on `stream` without host synchronisation; allocates and frees about
 * 5.1 * n * nev * 8 bytes of workspace stream-ordered (13 GB at n = 32768,
 * nev = 9830). The cost of a cluster of m eigenvalues grows as m^2 n.
 * Errors: TBBT_EINVAL (n < 0, nev outside [0, n], ldx < max(1, n), xtype,
 * null or misaligned pointers when there is work), TBBT_ENOMEM, TBBT_ECUDA.
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_tridiag_eig(const double *d, const double *e, int64_t n, int64_t nev, double *w, void *x,
                             int64_t ldx, tbbt_dtype xtype, void *stream);

/* -------------------------------------------------------------------------
 * Band -> full back-transformation of eigenvectors (Eq. 6e, Sec. 2.1):
 * C = P^* Y = Q1 Y, Q1 = H_0 H_1 ... H_{K1-1}, K1 = max(n - nbw, 0), the
 * reflectors of the full -> band reduction (Eq. 6a). Reflector c acts on rows
 * c+nbw .. n-1: H_c = I - tau[c] v_c v_c^H with v_c[c+nbw] = 1 (not stored)
 * and v_c[c+nbw+1 : n] = a[c+nbw+1 : n, c] (LAPACK layout: the reflectors sit
 * below the band of the reduced matrix; entries at or above the nbw-th
 * sub-diagonal are not read).
 *
 * a:    device, n x n column-major, lda >= max(1, n); read only.
 * tau:  device, K1 entries; read only.
 * q:    device, n x nev column-major, ldq >= max(1, n); in: Y (the
 *       eigenvectors of the band matrix, e.g. the output of
 *       tbbt_trans_ev_tridi_to_band_*), out: C. Columns are independent.
 * Complex variant: a, tau and q are interleaved complex128.
 * Runs on `stream` (NULL: the legacy default stream) without host
 * synchronisation; allocates and frees a P x 32 x 32 workspace of T factors
 * stream-ordered (P = ceil(K1/32)). Any nbw >= 1; nbw >= n is a no-op.
 * Errors: TBBT_EINVAL for n < 0, nbw < 1, nev outside [0, n], small lda/ldq,
 * null or misaligned pointers when there is work; TBBT_ENOMEM, TBBT_ECUDA.
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_trans_ev_band_to_full_d(const double *a, int64_t lda, const double *tau, int64_t n, int64_t nbw,
                                         int64_t nev, double *q, int64_t ldq, void *stream);
tbbt_status tbbt_trans_ev_band_to_full_z(const void *a, int64_t lda, const void *tau, int64_t n, int64_t nbw,
                                         int64_t nev, void *q, int64_t ldq, void *stream);

/* -------------------------------------------------------------------------
 * Band -> full back-transformation, split-precision form on the tensor cores
 * (Eq. 6e, real data): the same result as tbbt_trans_ev_band_to_full_d, with
 * the 32-reflector WY blocks I - V T V^T applied as Y <- Y - U (V^T Y),
 * U = V T, by exact products of 8-bit digit slices on BF16 tensor cores
 * (tcgen05): Y in 64-bit fixed point per column (exponent from the column's
 * norm), V and U in 6 digits scaled per block and per row, W = V^T Y summed
 * in 64-bit integers across 96-row batches and across the CTAs that share a
 * 128-column strip. Error: a few units of 2^-48 of a column's norm per
 * block, in practice ~1e-14 absolute on unit-norm columns.
 *
 * Arguments, layouts, ownership and the reflector store as for
 * tbbt_trans_ev_band_to_full_d. Needs a GPU of compute capability 10.x
 * (TBBT_ENOTSUP otherwise) and a cooperative launch of one CTA per SM.
 * Allocates stream-ordered workspace of about 24 * n^2 / 2 bytes of digit
 * slices plus 8 * n * nev bytes for the fixed-point Y (13 GB + 2.6 GB at
 * n = 32768, nev = 9830). A wait between CTAs that exceeds 20 s records
 * TBBT_ETIMEOUT (tbbt_stream_check reports it).
 * Errors: as tbbt_trans_ev_band_to_full_d, plus TBBT_ENOTSUP.
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_trans_ev_band_to_full_split_d(const double *a, int64_t lda, const double *tau, int64_t n,
                                               int64_t nbw, int64_t nev, double *q, int64_t ldq, void *stream);
/* The same with options. wait_timeout_ms: limit of each wait between CTAs
 * (0: 20000). debug_withhold_cta: test hook, -1 in normal use; otherwise the
 * CTA (strip-major: strip * S_K + slot) whose W publications are not
 * counted, so that the waits of its strip run out, TBBT_ETIMEOUT is recorded
 * and every CTA drains and exits (failure detection without a GPU fault).
 * Errors: as above, plus TBBT_EINVAL for wait_timeout_ms < 0 or
 * debug_withhold_cta < -1. */
tbbt_status tbbt_trans_ev_band_to_full_split_opts_d(const double *a, int64_t lda, const double *tau, int64_t n,
                                                    int64_t nbw, int64_t nev, double *q, int64_t ldq,
                                                    int32_t wait_timeout_ms, int32_t debug_withhold_cta,
                                                    void *stream);

/* -------------------------------------------------------------------------
 * FP64 rate probe (a measurement aid; the paper has no counterpart). The
 * FP64 back-transformation is bound by the FP64 pipe, so its roofline
 * denominator is that pipe's rate, measured on the device in use:
 * kind 0 launches `blocks` x `threads` threads that each run 8 independent
 * FP64 FMA chains for `iters` iterations; kind 1 runs, per warp, 4
 * independent FP64 tensor-core products (mma.sync m8n8k4) for `iters`
 * iterations. *flops receives the launch's flop count (2 per FMA, 512 per
 * m8n8k4 product); time the launch with events on `stream`.
 * d_sink: device array of blocks * threads doubles (written, meaningless).
 * Errors: TBBT_EINVAL (kind, threads not a multiple of 32 in [32, 1024],
 * blocks < 1, iters < 1, null pointers), TBBT_ECUDA.
 * ------------------------------------------------------------------------- */
tbbt_status tbbt_fp64_probe(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, double *d_sink,
                            double *flops, void *stream);

/* Host-side check of the block schedule (no GPU needed): largest number of
 * rows a thread block ever holds at once for these parameters, or -1 if the
 * schedule would touch a row twice in one step. Used by tests to show the
 * shared-memory ring never wraps onto live rows. */
int64_t tbbt_schedule_max_live_rows(int64_t n, int64_t nbw, int is_complex, int32_t sweeps_per_block,
                                    int32_t stages_per_step);

/* Host-side check of the split band -> full form's layout (no GPU needed):
 * for these sizes and an SM count, walks the layout the launcher of
 * tbbt_trans_ev_band_to_full_split_d would use, as its kernels walk it, and
 * returns 0 if every row of every 32-reflector block belongs to exactly one
 * (slot, batch, part) row of both the apply and the preparation kernel, each
 * (strip, slot) has exactly one CTA, and each block's counter target is its
 * number of slots with rows; a negative code names the first failed check
 * (-1: bad arguments). *slots_per_strip and *items (nullable) receive the
 * slots per 128-column strip and the number of (block, slot, batch) items. */
int64_t tbbt_b2f_split_layout_check(int64_t n, int64_t nbw, int64_t nev, int32_t sms, int32_t *slots_per_strip,
                                    int64_t *items);

#ifdef __cplusplus
}
#endif

#endif /* TBBT_H */
