/*
 * fftalign.h -- C ABI of libfftalign.so: GB300 (sm_103a) kernels for the
 * O(N log N) FFT-based rigid alignment of closed planar curves
 * (Dogan, Bernal & Hagwood, "FFT-based Alignment of 2d Closed Curves with
 * Application to Elastic Shape Analysis", arXiv 2501.17779).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Curves.  A curve is a list of n DISTINCT nodes p_0..p_{n-1} in counter-
 *   clockwise order; closure is implicit (the paper lists N points with first
 *   = last, Sec. 2, i.e. N-1 distinct nodes).  Points are interleaved doubles
 *   (x0, y0, x1, y1, ...) -- numpy/torch complex128 layout -- or, where a
 *   function says so, interleaved floats (complex64 layout).
 * Shift.  shift s in [0, N) is the cyclic start point t0 = s/N of Eq. energy:
 *   curve 2 is read at node k+s (mod N).  (The paper's m = s+1, t0 = t_m.)
 * Angle.  theta is the COUNTER-clockwise angle of the optimal rotation applied
 *   to curve 2, in (-pi, pi]: e^{i theta} z2[(k+s) mod N] best matches z1[k].
 *   The paper's R(theta) (Sec. 2) is clockwise, so its theta is -theta here.
 * Energy.  E = h sum_k |z1[k] - e^{i theta} z2[(k+s) mod N]|^2, h = 1/N
 *   (Eq. disc-energy, uniform trapezoid rule over the N distinct nodes).
 * Memory.  Every array argument is a DEVICE pointer owned by the caller unless
 *   the function says otherwise.  Calls are asynchronous on `stream` (a
 *   cudaStream_t passed as void*; NULL is the legacy default stream) and
 *   return once the work is enqueued.  The library keeps no state outside the
 *   handle; a handle is tied to one device.
 * Errors.  Entry points return FA_OK (0) or a negative FA_ERR_* code and
 *   never abort or trap.  fa_last_error() gives a message for the calling
 *   thread's last failure.  Problems with one item's DATA never fail a call:
 *   they set that item's status byte and write NaN outputs for it.
 */
#ifndef FFTALIGN_H
#define FFTALIGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fa_handle fa_handle;

/* return codes */
#define FA_OK 0
#define FA_ERR_INVALID_ARG (-1) /* null pointer, negative count, bad enum      */
#define FA_ERR_UNSUPPORTED (-2) /* size outside the supported set              */
#define FA_ERR_CUDA (-3)        /* CUDA runtime error (message in fa_last_error) */
#define FA_ERR_WORKSPACE (-4)   /* caller workspace smaller than required      */

/* per-item status bytes */
#define FA_STATUS_OK 0
#define FA_STATUS_DEGENERATE 1 /* fewer than 4 nodes, a zero-length segment,
                                  zero perimeter                               */
#define FA_STATUS_NONFINITE 2  /* a NaN or Inf coordinate in the input        */
#define FA_STATUS_BAD_SIZE 3   /* node count outside the supported range       */

/* resampling flags */
#define FA_CENTER 1      /* subtract the mean of the N resampled nodes         */
#define FA_UNIT_LENGTH 2 /* divide by the closed-polygon perimeter of the nodes */
#define FA_STORE_FP32 4  /* write complex64 (float2) instead of complex128     */

/* storage type of aligned curves */
#define FA_Z_F64 0 /* complex128: interleaved doubles */
#define FA_Z_F32 1 /* complex64: interleaved floats (widened to FP64 on load) */

/* alignment method */
#define FA_FFT 0    /* Algorithm 2 with the convolution theorem: O(N log N)   */
#define FA_DIRECT 1 /* every shift by its O(N) definition: O(N^2) baseline    */

/* arithmetic of the shift search (theta and the energy have FP64 accuracy) */
#define FA_PREC_FP64 0  /* every step in FP64                                  */
#define FA_PREC_MIXED 1 /* FA_FFT only: the three transforms in double-float
                           arithmetic (pairs of floats, ~48-bit significands)
                           on the FP32 pipe; their error (~1e-13 of max|c|)
                           keeps the argmax inside the tie tolerance; c(s*),
                           theta and the energy are computed in FP64, so the
                           result obeys the same bounds as FA_PREC_FP64.
                           Coordinates must lie within [2^-74, 2^128) in
                           magnitude (or be 0): unit-length curves do        */
/* fa_align_all_pairs only, N = 256 or 512: the search as a dense GEMM on the
 * tensor cores (tcgen05; the DFT of every cross-spectrum Z_i conj(Z_j), Sec. 2),
 * float32 accumulation, the 8 shifts of largest |c|^2 kept per pair, those 8
 * re-scored by their direct correlation in double-float arithmetic (~1e-14),
 * theta and the energy at the winner likewise (FP64-bound accuracy).  The
 * operands enter the tensor core as:                                        */
#define FA_PREC_TC_BF16X3 2 /* bfloat16 hi + lo pieces, 3 products (~16 bits) */
#define FA_PREC_TC_FP16X3 3 /* float16 hi + lo pieces, 3 products (~22 bits)  */
#define FA_PREC_TC_TF32 4   /* one TF32 product (~11 bits)                     */
#define FA_PREC_TC_TF32X3 5 /* TF32 hi + lo pieces, 3 products (~21 bits)      */
/* A pair whose best shift lies outside its 8 candidates gets the best of
 * them: the reduced operand precision decides how often that happens (the
 * tests and the benchmark report the agreement with FA_PREC_FP64).           */

/* key types of fa_select_k */
#define FA_KEY_F32 0
#define FA_KEY_F64 1

/* Create a handle bound to CUDA device `device` (its twiddle tables are built
 * here, synchronously).  *h receives the handle.  Not thread-safe with
 * respect to the same handle being destroyed concurrently. */
int fa_create(fa_handle** h, int device);

/* Release a handle and the device memory it owns.  Waits for nothing: the
 * caller must make sure no work that uses the handle is still in flight. */
int fa_destroy(fa_handle* h);

/* Message for the calling thread's last non-zero return code (static
 * storage, thread-local; "" if none). */
const char* fa_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int fa_version(void);

/*
 * Arc-length resampling (Sec. 2: Eq. arc-length-param, then cubic-spline
 * interpolation at uniform parameters t_k = k/N_out).
 *
 * For each of C curves given in CSR form -- nodes pts[offsets[i] ..
 * offsets[i+1]) -- the knot of node l is its cumulative chord length divided
 * by the closed-polygon perimeter (u_0 = 0, u_n = 1 closing the curve), a
 * periodic C2 cubic spline is fitted through (u_l, p_l) for x and y, and it
 * is evaluated at t_k = k/N_out, k = 0..N_out-1.  With FA_CENTER the node
 * mean of the N_out outputs is subtracted; with FA_UNIT_LENGTH the outputs
 * are divided by their closed-polygon perimeter (applied after centring).
 * An explicit closing duplicate (last node == first node) is ignored.
 *
 *   pts        double[2*n_pts]  interleaved x,y of all curves (device)
 *   offsets    int64[C+1]       CSR offsets, non-decreasing, offsets[C] <= n_pts (device)
 *   C          number of curves (>= 0)
 *   n_pts      length of pts in points (>= offsets[C]); sizes the workspace
 *   N_out      nodes per resampled curve, in [4, 1<<20]
 *   flags      FA_CENTER | FA_UNIT_LENGTH | FA_STORE_FP32
 *   z_out      [C][N_out] complex128, or complex64 with FA_STORE_FP32 (device)
 *   status     int8[C] per-curve status (device): FA_STATUS_OK, _DEGENERATE
 *              (fewer than 4 distinct nodes, a repeated node, zero perimeter),
 *              _NONFINITE, or _BAD_SIZE (the kernel checks each curve's
 *              offsets: a range that runs backwards, starts below 0, ends
 *              beyond n_pts or holds more than 2^30 nodes is skipped, so that
 *              a bad CSR array never reads or writes outside pts and the
 *              workspace); the curve's outputs are NaN unless OK
 *   workspace  device scratch of at least fa_resample_workspace_size() bytes,
 *              256-byte aligned, or NULL to let the handle provide it (the
 *              handle's buffer then grows with cudaMalloc when needed, and
 *              calls on different streams sharing one handle must not overlap)
 */
size_t fa_resample_workspace_size(int64_t C, int64_t n_pts, int32_t N_out, int32_t flags);
int fa_resample_arclength(fa_handle* h, const double* pts, const int64_t* offsets, int64_t C,
                          int64_t n_pts, int32_t N_out, int32_t flags, void* z_out,
                          int8_t* status, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Rigid alignment of P pairs (Algorithm 2; Algorithm 1 in closed form).
 *
 * Pair p is z1[p][0..N) and z2[p][0..N), both assumed centred and of unit
 * length (Sec. 2).  For every shift s the optimal rotation has the closed form
 * theta(s) = arg c(s) with the cyclic cross-correlation
 *     c(s) = sum_k z1[k] conj(z2[(k+s) mod N]),
 * the complex form of A(t_m) in Eq. A-mtx (Re c = A11 + A22, Im c = A21 - A12),
 * and max over R of tr(R A^T) = |c(s)|, so the best shift maximises |c(s)|.
 * FA_FFT evaluates c for all s with three FFTs (forward transforms of z1 and
 * z2, then c = DFT(Z1 * conj(Z2)) / N -- the convolution theorem of Sec. 2);
 * FA_DIRECT evaluates the O(N) sum for every s (the O(N^2) search the paper
 * compares against).  Exact ties go to the smallest s.  At the winning shift
 * c(s*) is recomputed by its O(N) sum, theta = atan2(Im c, Re c) and the
 * energy is evaluated directly from its definition (no cancellation).
 *
 *   z1, z2   [P][N] complex128 (FA_Z_F64) or complex64 (FA_Z_F32) (device)
 *   P        number of pairs (>= 0)
 *   N        nodes per curve: a power of two in [4, 4096] for FA_FFT,
 *            any value in [1, 4096] for FA_DIRECT
 *   ztype    FA_Z_F64 | FA_Z_F32
 *   method   FA_FFT | FA_DIRECT
 *   prec     FA_PREC_FP64, or FA_PREC_MIXED with FA_FFT
 *   shift    int32[P]   best shift (-1 when status != 0)
 *   theta    double[P]  CCW angle applied to curve 2 (NaN when status != 0)
 *   energy   double[P]  energy at the optimum (NaN when status != 0)
 *   status   int8[P]    FA_STATUS_OK or FA_STATUS_NONFINITE
 */
int fa_align_pairs(fa_handle* h, const void* z1, const void* z2, int64_t P, int32_t N,
                   int32_t ztype, int32_t method, int32_t prec, int32_t* shift, double* theta,
                   double* energy, int8_t* status, void* stream);

/*
 * All-pairs alignment matrix of M curves (Algorithm 2 for every ordered pair).
 *
 * Entry (i, j) is the alignment of curve j onto curve i, i.e. fa_align_pairs
 * with z1 = curve i and z2 = curve j: shift[i*M + j], theta[i*M + j],
 * energy[i*M + j].  Each curve's spectrum is computed once into the
 * workspace; the pairs i < j are searched (one transform per pair) and the
 * pair (j, i) follows from the symmetry of the energy: shift (N - s) mod N,
 * angle -theta, the same energy (on exact ties this may differ from a
 * direct search of (j, i), which would report its own smallest shift).  The
 * diagonal is shift 0, angle 0, energy 0.
 *
 *   z          [M][N] complex128 (FA_Z_F64) or complex64 (FA_Z_F32) (device),
 *              centred and of unit length
 *   M          number of curves, in [0, 65536]
 *   N          nodes per curve, a power of two in [4, 4096]
 *   prec       FA_PREC_FP64, FA_PREC_MIXED (search in double-float) or
 *              FA_PREC_TC_* (search on the tensor cores, N = 256 or 512 and
 *              2 <= M: the workspace is then
 *              fa_align_all_pairs_workspace_size_prec(M, N, prec) bytes)
 *   shift      int32[M*M], theta double[M*M], energy double[M*M] (device)
 *   status     int8[M] per-curve status (FA_STATUS_OK or _NONFINITE); rows and
 *              columns of a non-finite curve get shift -1 and NaN
 *   workspace  device scratch of fa_align_all_pairs_workspace_size(M, N)
 *              bytes (M*N*16), 256-byte aligned, or NULL for the handle's
 */
size_t fa_align_all_pairs_workspace_size(int64_t M, int32_t N);
/* workspace of fa_align_all_pairs for a given precision: M*N*16 bytes for
 * FA_PREC_FP64 and FA_PREC_MIXED; for FA_PREC_TC_* the spectra in FP64 and
 * complex64, the split DFT matrix (4 MB at N = 512) and 16 bytes per ordered
 * pair for the candidates (M*M*16); 0 for unsupported arguments */
size_t fa_align_all_pairs_workspace_size_prec(int64_t M, int32_t N, int32_t prec);
int fa_align_all_pairs(fa_handle* h, const void* z, int64_t M, int32_t N, int32_t ztype,
                       int32_t prec, int32_t* shift, double* theta, double* energy,
                       int8_t* status, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Elastic shape distance (Sec. 3): for each pair p, curve idx1[p] of set 1
 * against curve idx2[p] of set 2, the minimum over (t0, R, gamma) of
 * Eq. dist2-energy, E = int |R q1(t + t0) - sqrt(gamma') q2(gamma(t))|^2 dt,
 * with q = beta'/|beta'|^{1/2} the SRV functions of the unit-length curves,
 * by "Approach 2" started from the FFT pre-alignment (Sec. 3): the curves are
 * resampled in arc length and rigidly aligned (Algorithm 2, motion on curve
 * 1); then gamma-steps and (t0,R)-steps (Algorithm 2 applied to SRV
 * functions, without resampling) alternate until an iteration lowers E by at
 * most 1e-12 or max_iter iterations have run.  The gamma-step is this
 * library's own (the paper takes it from a reference it does not state): a
 * dynamic programme over lattice paths with steps (a,b), a,b <= 3, coprime,
 * in the band |i - j| <= band, run when the start point changed, followed by
 * 16 Levenberg-Marquardt steps on gamma's node values, its offset and theta.
 *
 * Discretisation: a curve is N nodes, node k at parameter k/N (its own
 * parameterisation, not resampled), closed, scaled to unit polygon length;
 * q is sampled at the cell midpoints from the chords and read between samples
 * by the periodic Catmull-Rom cubic; gamma is piecewise linear with node
 * values g_k = N gamma(k/N), g_N = g_0 + N; E is taken by the midpoint rule.
 *
 *   curves1    [M1][N] complex128 (device): set 1 (moved by (t0, R))
 *   curves2    [M2][N] complex128 (device): set 2 (reparameterised by gamma)
 *   N          nodes per curve, a power of two in [32, 1024] (with fewer nodes the
 *              iteration is not stable under rounding)
 *   idx1, idx2 int64[P] (device) curve indices into the sets, or NULL for
 *              pair p = (p, p) (then M1, M2 >= P); an index out of range gives
 *              status FA_STATUS_BAD_SIZE for that pair
 *   band       half-width B of the lattice band, -1 (or >= N) for the full
 *              lattice; the refinement is not confined to it
 *   max_iter   iterations at most, in [0, 1000]; 0 runs none and returns the
 *              starting triple: the pre-alignment's shift and angle, the lattice
 *              path of the first gamma-step (its path sums are float32: it only
 *              picks where the refinement starts) in gamma, and that triple's
 *              FP64 energy, with iters = 0
 *   shift      int32[P]   s, t0 = s/N (-1 when status != 0)
 *   theta      double[P]  CCW angle of R applied to curve 1 (NaN when status != 0)
 *   energy     double[P]  E of the final triple (the distance is sqrt(E))
 *   gamma      double[P][N+1] node values g_k, or NULL
 *   iters      int32[P]   iterations run, or NULL
 *   lm_steps   int32[P]   Levenberg-Marquardt steps taken by the gamma-steps
 *              (their sum over the iterations; the unit of most of the FP64
 *              work, for throughput accounting), or NULL
 *   status     int8[P]    FA_STATUS_OK, _DEGENERATE (a curve of zero length or
 *              fewer than 4 distinct nodes), _NONFINITE, _BAD_SIZE
 *   workspace  device scratch of fa_elastic_workspace_size(h, M1, M2, P, N, band)
 *              bytes, 256-byte aligned, or NULL for the handle's own
 * Returns FA_OK, FA_ERR_INVALID_ARG, FA_ERR_UNSUPPORTED, FA_ERR_WORKSPACE or
 * FA_ERR_CUDA.  Asynchronous on stream; graph-capturable when a workspace is
 * passed.
 */
size_t fa_elastic_workspace_size(fa_handle* h, int64_t M1, int64_t M2, int64_t P, int32_t N,
                                 int32_t band);
int fa_elastic_distance(fa_handle* h, const double* curves1, int64_t M1, const double* curves2,
                        int64_t M2, int32_t N, const int64_t* idx1, const int64_t* idx2,
                        int64_t P, int32_t band, int32_t max_iter, int32_t* shift,
                        double* theta, double* energy, double* gamma, int32_t* iters,
                        int32_t* lm_steps, int8_t* status, void* workspace,
                        size_t workspace_bytes, void* stream);

/*
 * Alignment of P pairs with DIFFERENT node counts, one persistent launch per
 * transform-length bucket.
 *
 * Pair p is z1[offsets[p] .. offsets[p+1]) and z2[offsets[p] .. offsets[p+1])
 * (n_p nodes each, same CSR offsets for both curves), otherwise as in
 * fa_align_pairs.  Any n_p in [4, max_n] is supported (max_n <= 8192): for a
 * power of two the transforms have length n_p; otherwise the cyclic
 * correlation is computed exactly as a zero-padded linear correlation with
 * transforms of length L = the power of two >= 2 n_p (no chirps, no
 * approximation).  The pairs are sorted on the device into buckets by
 * transform length (log2 L, longest first); each bucket is processed by one
 * persistent launch with the handle's plan for that bucket -- the CTA size
 * and the number of pairs one CTA transforms side by side (several short
 * pairs per CTA for L <= 1024, one pair per CTA split into radix-R parts for
 * L > 4096) -- whose CTAs take pairs from the bucket's counter.  The plans
 * start from a size rule and are set per bucket by
 * fa_align_pairs_ragged_autotune.  Every step is a launch or memset on
 * `stream`, so the call can be captured into a CUDA graph (pass a workspace
 * then, so that nothing is allocated).
 *
 *   z1, z2     complex128 (FA_Z_F64) or complex64 (FA_Z_F32) arrays of
 *              offsets[P] points (device), each curve centred, unit length
 *   offsets    int64[P+1] non-decreasing CSR offsets (device)
 *   max_n      upper bound on every n_p, in [4, 8192]; sizes the workspace;
 *              pairs with n_p < 4 or n_p > max_n get FA_STATUS_BAD_SIZE
 *   shift, theta, energy, status   as in fa_align_pairs ([P] each, device)
 *   workspace  fa_align_pairs_ragged_workspace_size(h, P, max_n) bytes,
 *              256-byte aligned, or NULL for the handle's buffer
 */
size_t fa_align_pairs_ragged_workspace_size(fa_handle* h, int64_t P, int32_t max_n);
int fa_align_pairs_ragged(fa_handle* h, const void* z1, const void* z2, const int64_t* offsets,
                          int64_t P, int32_t max_n, int32_t ztype, int32_t* shift, double* theta,
                          double* energy, int8_t* status, void* workspace, size_t workspace_bytes,
                          void* stream);

/*
 * Autotuner of fa_align_pairs_ragged: for every transform-length bucket the
 * caller's batch fills, runs that bucket's pairs with each compiled plan that
 * fits the length (CTA sizes 128..1024 threads, 1..16 pairs per CTA, and for
 * L = 8192 and 16384 also one pair per thread-block cluster of L/4096 CTAs),
 * one warm-up and three timed runs each, and keeps the fastest plan per bucket in
 * the handle for later calls (fa_align_pairs_ragged_plan reports them).
 * *chosen_threads receives the CTA size chosen for the longest bucket
 * present.  Same arguments and outputs as fa_align_pairs_ragged (the outputs
 * hold the chosen plans' result afterwards; different plans sum in a
 * different order and may differ in the last bit).  Synchronises the stream;
 * not for use during stream capture.
 */
int fa_align_pairs_ragged_autotune(fa_handle* h, const void* z1, const void* z2,
                                   const int64_t* offsets, int64_t P, int32_t max_n,
                                   int32_t ztype, int32_t* shift, double* theta, double* energy,
                                   int8_t* status, void* workspace, size_t workspace_bytes,
                                   void* stream, int32_t* chosen_threads);

/* The handle's plan for fa_align_pairs_ragged, per bucket b = log2 L in
 * [0, 16): threads[b] (CTA size), pairs_per_cta[b] (-R for one pair per
 * cluster of R CTAs), and ms[b], the time of
 * that bucket's launch measured by the last autotuning (0 when not tuned);
 * entries outside the supported lengths are 0.  Any pointer may be NULL
 * (HOST arrays of 16 entries). */
int fa_align_pairs_ragged_plan(fa_handle* h, int32_t* threads, int32_t* pairs_per_cta, float* ms);
/* Sets the handle's plan for bucket log2 L = bucket (in [2, 14]): one of the
 * compiled (threads, pairs_per_cta) combinations -- (256|512|1024, 1),
 * (128|256|512, 2), (128|256|512, 4), (256, 8), (256, 16), and the cluster
 * plans (256|512, -2) for L = 8192 and (256|512, -4) for L = 16384, in which
 * the R CTAs of a thread-block cluster share one pair (each transforms one of
 * the R decimation-in-frequency parts in its shared memory and the
 * recombination reads the others' parts through distributed shared memory)
 * -- that fits the length (pairs_per_cta >= 2 needs pairs_per_cta L <= 2048
 * and at most L threads per pair); FA_ERR_UNSUPPORTED otherwise. */
int fa_align_pairs_ragged_set_plan(fa_handle* h, int32_t bucket, int32_t threads,
                                   int32_t pairs_per_cta);

/*
 * End-to-end convenience call on HOST buffers: arc-length resampling of 2P
 * raw curves to N nodes (centred, unit length; fa_resample_arclength), then
 * rigid alignment of curve p with curve P+p (fa_align_pairs).
 *
 *   pts, offsets  HOST arrays: CSR of 2P curves, offsets[0] = 0; curves
 *                 0..P-1 are the first members of the pairs, P..2P-1 the
 *                 second.  Pinned (page-locked) memory gives asynchronous
 *                 copies; pageable memory works but copies synchronously.
 *   N             resampled nodes per curve (a power of two in [4, 4096] for
 *                 FA_FFT, [4, 4096] for FA_DIRECT)
 *   flags         0 or FA_STORE_FP32 (the resampled curves are kept as
 *                 complex64 between the two steps)
 *   method, prec  as for fa_align_pairs
 *   shift, theta, energy, status   HOST arrays of P entries; a pair whose
 *                 curve fails resampling gets that curve's status and NaNs
 *
 * For P >= 1024 the pairs run in two or four chunks, each on one of the
 * handle's own streams (upload of its curves, resampling, alignment,
 * download), so that uploads overlap the kernels; the caller's stream waits
 * for all of them.  Uses the handle's device buffer (grown with cudaMalloc
 * when needed), so calls sharing a handle must not run concurrently.  Returns
 * after the results are in the host arrays (the stream is synchronised).
 */
int fa_align_curves_host(fa_handle* h, const double* pts, const int64_t* offsets, int64_t P,
                         int32_t N, int32_t flags, int32_t method, int32_t prec, int32_t* shift,
                         double* theta, double* energy, int8_t* status, void* stream);

/*
 * Arc-length resampling that allocates nothing (the paper has no counterpart:
 * this is a deployment variant of fa_resample_arclength).
 *
 * For callers that cannot call cudaMalloc -- host applications that reserve
 * all device memory up front and do not let libraries allocate, and
 * latency-critical loops that cannot afford the implicit synchronisation of an
 * allocation.  Such callers cannot create a handle either (fa_create
 * allocates), so this call takes none and runs on the CURRENT device.  It
 * computes exactly what fa_resample_arclength computes, with the same
 * arguments except the handle and the workspace.
 *
 * Scratch: a fixed device array of FA_NOALLOC_SCRATCH_BYTES (64 MiB) that
 * every GPU which loads the library holds until the process exits.  A batch
 * needs fa_resample_workspace_size(C, n_pts, N_out, flags) bytes of it (48
 * bytes per input node, plus 16 bytes per output node with FA_STORE_FP32:
 * about 1.39 million input nodes per call); larger batches are rejected with
 * FA_ERR_UNSUPPORTED and a message giving both sizes.  Nothing is allocated
 * or freed; each call resets one 8-byte work counter inside the array with a
 * memset on `stream`.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device) and keeps it for the life of the
 * process; make that first call before any stream capture.  Calls after a
 * cudaDeviceReset of that device are not supported (the cached address
 * belongs to the context that was torn down).  All calls share the one array and it keeps the last call's
 * contents (every value a call reads it has written itself first): calls
 * whose work overlaps on the GPU -- on different streams, or from different
 * host threads -- race on it and must be serialised by the caller.
 */
#define FA_NOALLOC_SCRATCH_BYTES (64u << 20)
int fa_resample_arclength_noalloc(const double* pts, const int64_t* offsets, int64_t C,
                                  int64_t n_pts, int32_t N_out, int32_t flags, void* z_out,
                                  int8_t* status, void* stream);

/* ------------------------------------------------------------------------
 * k-NN retrieval under the elastic distance with learned candidate pruning.
 * Not part of the paper (Sec. 3 defines the distance); the pruning network is
 * this library's addition, with fa_elastic_distance as its fallback and as
 * the measure of its recall.
 * ---------------------------------------------------------------------- */

/*
 * Rotation-, translation- and cyclic-shift-invariant descriptors of curves
 * resampled uniformly in arc length (e.g. by fa_resample_arclength): with
 * Z = DFT(z)/N, out[m][f-1] = log(|Z[f]| + 1e-30) and out[m][F+f-1] =
 * log(|Z[-f]| + 1e-30) for f = 1..F.
 *   z    [M][N] complex128 (device), N a power of two in [8, 1024]
 *   out  float [M][2F] (device), 1 <= F < N/2
 */
int fa_fourier_descriptors(fa_handle* h, const double* z, int64_t M, int32_t N, int32_t F,
                           float* out, void* stream);

/* Column means and reciprocal population standard deviations of X [M][D]
 * (device, M > 0; a constant column gets 1/std = 1), and the in-place
 * standardisation X = (X - mean) * inv_std. */
int fa_column_stats(fa_handle* h, const float* X, int64_t M, int32_t D, float* mean,
                    float* inv_std, void* stream);
int fa_standardize(fa_handle* h, float* X, int64_t M, int32_t D, const float* mean,
                   const float* inv_std, void* stream);

/* out[q][g] = sum_d (A[q][d] - B[g][d])^2, float32 (device arrays), Q <= 2^21. */
int fa_embed_sqdist(fa_handle* h, const float* A, int64_t Q, const float* B, int64_t G,
                    int32_t D, float* out, void* stream);

/*
 * Per row of keys [rows][C] (float32 or float64 by key_type, device): the
 * positions of the k smallest keys, ascending by (key, position) (NaN last),
 * into out_pos [rows][k]; their keys into out_keys [rows][k] (same type) when
 * not NULL.  1 <= k <= min(256, C).
 */
int fa_select_k(fa_handle* h, const void* keys, int32_t key_type, int64_t rows, int64_t C,
                int32_t k, int64_t* out_pos, void* out_keys, void* stream);

/*
 * The pruning network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, dimensions
 * 64 -> 256 -> 256 -> 64, weights used in bfloat16 (float32 master values),
 * biases, activations and accumulation in float32.  Parameters are one flat
 * float32 vector of fa_mlp_num_params() values: W1 [256][64], b1 [256],
 * W2 [256][256], b2 [256], W3 [64][256], b3 [64], each row-major.
 *
 * fa_mlp_create      He-normal weights from seed (SplitMix64, Box-Muller), the
 *                    output layer's scaled by 0.01, zero biases; the handle owns device memory and must be
 *                    released with fa_mlp_destroy.
 * fa_mlp_set_params  copies a host parameter vector in (and zeroes the Adam
 *                    state); fa_mlp_get_params copies it out (synchronous).
 * fa_mlp_forward     Y [B][64] = network(X [B][64]) (device arrays), B <= 2^21.
 * fa_mlp_pair_grad   for pairs p: rows pi[p], pj[p] of X [rows][64] (device),
 *                    target distances d [P] (float32, device): the loss
 *                    L = (1/P) sum_p (r_p - d_p)^2 / (d_p + 0.05)^2,
 *                    r_p = sqrt(|y_pi - y_pj|^2 + 1e-12), into *loss (device
 *                    float), and dL/dparams into the handle (and into grad
 *                    [fa_mlp_num_params()] on the device when not NULL);
 *                    P <= 2^20.
 *                    Synchronises the stream; an index outside [0, rows)
 *                    returns FA_ERR_INVALID_ARG.
 * fa_mlp_adam_step   one Adam step (0.9, 0.999, 1e-8) with learning rate lr
 *                    from the last gradient; refreshes the bfloat16 copy.
 */
typedef struct fa_mlp fa_mlp;
int64_t fa_mlp_num_params(void);
int fa_mlp_create(fa_handle* h, uint64_t seed, fa_mlp** out);
int fa_mlp_destroy(fa_mlp* m);
int fa_mlp_set_params(fa_mlp* m, const float* params);
int fa_mlp_get_params(fa_mlp* m, float* params);
int fa_mlp_forward(fa_mlp* m, const float* X, int64_t B, float* Y, void* stream);
int fa_mlp_pair_grad(fa_mlp* m, const float* X, int64_t rows, const int64_t* pi,
                     const int64_t* pj, const float* d, int64_t P, float* loss, float* grad,
                     void* stream);
int fa_mlp_adam_step(fa_mlp* m, float lr, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFTALIGN_H */
