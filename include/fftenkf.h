/*
 * fftenkf.h - C ABI of the GB300 FFT Ensemble Kalman Filter analysis step.
 *
 * Method: Mandel, Beezley, Kondratenko, "Fast Fourier Transform Ensemble Kalman
 * Filter with Application to a Coupled Atmosphere-Wildland Fire Model",
 * Sec. 2.1.  Every member is transformed by the 2-D DFT F (step 1), the
 * forecast covariance is replaced by its frequency-domain diagonal
 *   chat_i = 1/(N-1) sum_k |uhat_ik - mean_k uhat_ik|^2              eq. (dii)
 * with the cross spectra of eq. (cov-multi-spectral) for a block state, and the
 * analysis is applied wavenumber by wavenumber
 *   uhat_k^(j),a = uhat_k^(j) + chat^(jo) (chat^(oo) + rhat_o)^-1
 *                  (dhat_o + ehat_{k,o} - uhat_k^(o))       eq. (spectral-multi-enkf)
 * i.e. as a convolution in physical space instead of a tapered sparse solve.
 *
 * Conventions (all calls):
 *  - Grids are ny x nx, doubly periodic, x fastest.  nx, ny in {2^a, 3*2^a};
 *    16 <= nx <= 8192 and 16 <= ny <= 4096.  F is the unitary DFT, so white
 *    noise of variance r has rhat == r (R = rI of Sec. 2.1).
 *  - Block state of Sec. 2.1 eq. (block-enkf): M = n_blocks fields, N = n_members
 *    members; observed_mask[j] != 0 marks H^(j) = I, all other H^(j) = 0.
 *    Mutual cross-covariances of distinct observed blocks are neglected (the
 *    rule Sec. 2.2 applies to the components of the morphed state): an
 *    observed block is corrected by its own innovation only, an unobserved
 *    block j by the sum over observed o of chat^(jo)/(chat^(oo)+rhat_o).
 *  - The cross spectrum is chat^(jo) = 1/(N-1) sum_k ahat_k^(j) conj(ahat_k^(o)),
 *    the frequency diagonal of the sample cross-covariance C_N^(jo).
 *  - Half spectrum tables are [ny][nx/2+1] (k_y = 0..ny-1, k_x = 0..nx/2).
 *  - Array arguments are DEVICE pointers owned by the caller, contiguous,
 *    16-byte aligned (workspace: 256-byte aligned); a violation returns
 *    FFTENKF_EINVAL before anything is launched.  Storage FFTENKF_BF16 arrays
 *    hold bfloat16 values, FFTENKF_F32 arrays float.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work and return without synchronising; only fftenkf_last_device_status
 *    waits for the stream.  Device-side failures (a non-finite covariance
 *    estimate) are recorded in the plan's status word, never trapped.
 *  - Calls on one plan must not overlap in time on different streams: the plan
 *    owns one auxiliary stream and its status word.
 */
#ifndef FFTENKF_H
#define FFTENKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFTENKF_OK = 0,
  FFTENKF_EINVAL = 1,        /* bad argument: null or misaligned pointer, bad dims */
  FFTENKF_EUNSUPPORTED = 2,  /* size not 2^a or 3*2^a in range, N < 2, too many blocks */
  FFTENKF_ECUDA = 3,         /* a CUDA runtime call failed */
  FFTENKF_ENONFINITE = 4,    /* non-finite spectral covariance seen on the device */
  FFTENKF_ETIMEOUT = 5,      /* a bounded device wait for an asynchronous copy gave up */
  FFTENKF_ENOMEM = 6         /* device allocation failed */
} fftenkf_status;

typedef enum { FFTENKF_F32 = 0, FFTENKF_BF16 = 1 } fftenkf_storage;

typedef struct {
  int ny, nx;        /* grid */
  int n_blocks;      /* M, 1..16 */
  int n_members;     /* N >= 2 (eq. dii divides by N-1) */
  int storage;       /* fftenkf_storage of ensemble and perturbations */
} fftenkf_dims;

typedef struct fftenkf_plan_s* fftenkf_plan;

/* Create a plan for one (dims, observed_mask).  observed_mask: HOST array of
 * n_blocks bytes.  The plan owns twiddle tables, a device status word and an
 * auxiliary stream; it allocates device memory (a few MB) here only.
 * Returns EUNSUPPORTED when the sizes or block counts are outside the limits
 * above or the per-wavenumber statistics do not fit in shared memory. */
fftenkf_status fftenkf_plan_create(fftenkf_plan* plan, const fftenkf_dims* dims,
                                   const uint8_t* observed_mask);
fftenkf_status fftenkf_plan_destroy(fftenkf_plan plan);

/* Bytes of device workspace estimate_spectrum / analyze need. */
fftenkf_status fftenkf_workspace_size(fftenkf_plan plan, size_t* bytes);

/* Number of doubles in a spectrum table set: n_obs*K real auto tables followed
 * by n_obs*n_unobs complex cross tables (2K doubles each), K = ny*(nx/2+1).
 * Order: chat^(oo) for observed o ascending; then for observed o ascending,
 * chat^(jo) for unobserved j ascending; complex values as (re, im) pairs. */
fftenkf_status fftenkf_spectrum_size(fftenkf_plan plan, size_t* n_doubles);

/* Steps 1-2 of Sec. 2.1 (eq. dii, eq. cov-multi-spectral): the spectral
 * covariance tables of `ensemble` ([M][N][ny][nx], storage dtype), unitary
 * scaling, written to spectrum_out (device, fftenkf_spectrum_size doubles).
 * No mean field is formed: the first member of every block is the pivot, the
 * differences u_k - u_0 are transformed (exact in FP32 for BF16 members, and for
 * FP32 members within a factor two of each other), and the products of the
 * transformed sum of those differences are subtracted from the accumulated ones,
 * which gives the same sample covariance.  Where the ensemble has no variance
 * above FFT round-off an auto table entry can then come out a few rounding
 * errors below 0.
 * workspace: device buffer of fftenkf_workspace_size bytes, or NULL to use a
 * buffer the plan allocates on first use and keeps. */
fftenkf_status fftenkf_estimate_spectrum(fftenkf_plan plan, const void* ensemble, double* spectrum_out,
                                         void* workspace, void* stream);

/* The analysis of eq. (spectral-multi-enkf), in place on `ensemble`
 * ([M][N][ny][nx], storage dtype; rounded to nearest even for BF16).
 *   data          [n_obs][ny][nx] float: d for every observed block (ascending)
 *   perturbations [N][n_obs][ny][nx] storage dtype: e_k ~ N(0, R) (Sec. 2)
 *   rhat          [n_obs][ny][nx/2+1] double: spectral data-error variance; it
 *                 must be even in k (rhat(-k) = rhat(k)), as the spectrum of a
 *                 real noise field is; where chat^(oo) + rhat == 0 the gain is 0
 *   spectrum      NULL: estimated from the ensemble (steps 1-2); otherwise a
 *                 caller-supplied table set in the fftenkf_spectrum_size layout
 *                 (e.g. a denoised or exact spectrum) used in place of chat.
 * The result is u + Re F^-1[...]; with a caller spectrum that is not
 * Hermitian-symmetric on the k_x = 0 and k_x = nx/2 columns the real part is
 * what is returned. */
fftenkf_status fftenkf_analyze(fftenkf_plan plan, void* ensemble, const float* data,
                               const void* perturbations, const double* rhat, const double* spectrum,
                               void* workspace, void* stream);

/* The same analysis with the perturbations e_{k,o} ~ N(0, R_o) drawn by the library
 * (eq. enkf: the EnKF's data perturbations; R_o = F* diag(rhat_o) F) instead of passed in:
 * in frequency space, ehat_{k,o} = sqrt(rhat_o) zhat_{k,o} with zhat the unitary DFT of a
 * white N(0, 1) field (Hermitian, real at the self-conjugate wavenumbers), added to the
 * innovation spectrum after its forward transform, so no perturbation field is stored or
 * read.  zhat comes from the counter-based generator Philox4x32-10 (Salmon et al., SC 2011)
 * with key `seed`: in the columns 0 < k_x < nx/2 the counter (k_y mod ny/2, k_x, k n_obs + o, 0)
 * serves k_y < ny/2 (words 0, 1) and k_y + ny/2 (words 2, 3); in the columns k_x = 0, nx/2 the
 * counter is (min(k_y, ny - k_y), k_x, k n_obs + o, 0), words 0, 1; Box-Muller on the top 24
 * bits of a word pair.  The same seed gives the same analysis.  Other arguments, layouts
 * and errors as fftenkf_analyze. */
fftenkf_status fftenkf_analyze_seeded(fftenkf_plan plan, void* ensemble, const float* data, const double* rhat,
                                      const double* spectrum, unsigned long long seed, void* workspace,
                                      void* stream);

/* Allocation-free estimate for one block (the paper has no counterpart: this
 * is a deployment variant of fftenkf_estimate_spectrum).  For callers that may
 * not call cudaMalloc -- e.g. a host framework that owns every device
 * allocation through its own pool, or a latency-critical loop that cannot
 * afford cudaMalloc's implicit synchronisation -- it needs no plan and no
 * workspace: all scratch (twiddle tables, row spectra, covariance table,
 * status word) comes from one static device array of 64 MiB that every GPU
 * loading this library holds until the process exits.  It allocates nothing
 * and calls no allocating routine.
 *   ensemble      [N][ny][nx] device array of the storage type (one block)
 *   spectrum_out  [ny][nx/2+1] device doubles: the same single-block table that
 *                 fftenkf_estimate_spectrum writes (unitary scaling)
 * Sizes follow the plan limits; a problem whose scratch exceeds the array
 * (about N (nx/2) ny 8 bytes plus small tables > 64 MiB) returns
 * FFTENKF_EUNSUPPORTED with a message giving the bytes needed.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it, so make that first call before any
 * stream capture.  All calls share the one array and it keeps the last call's
 * contents; calls that overlap on the GPU (on different streams, or from
 * different host threads) race on it and must be serialised by the caller.
 * Each call clears the array's status word before its kernels run; whether a
 * bounded wait gave up (the table then holds stale values) or a covariance value
 * was not finite is read with fftenkf_static_last_device_status. */
fftenkf_status fftenkf_estimate_spectrum_static(const void* ensemble, int ny, int nx, int n_members, int storage,
                                                double* spectrum_out, void* stream);

/* Status of the last fftenkf_estimate_spectrum_static calls on the current
 * device (the paper has no counterpart): waits for `stream`, reads and clears the
 * static array's status word without allocating, and returns FFTENKF_OK,
 * FFTENKF_ETIMEOUT (a bounded wait for a copy gave up: spectrum_out is stale),
 * FFTENKF_ENONFINITE (a covariance value was not finite), or FFTENKF_ECUDA if the
 * stream reported an error.  Reads before any call on the device return OK. */
fftenkf_status fftenkf_static_last_device_status(void* stream);

/* Wait for `stream`, then return and clear the plan's device status word:
 * FFTENKF_OK, FFTENKF_ETIMEOUT (a bounded wait for an asynchronous copy gave up;
 * the outputs of that call are incomplete), FFTENKF_ENONFINITE, or FFTENKF_ECUDA
 * if the stream reported an error. */
fftenkf_status fftenkf_last_device_status(fftenkf_plan plan, void* stream);

/* Test setting of the error path of the bounded waits: with on != 0, every CTA
 * of the forward anomaly row pass gives up its first wait for a bulk copy at
 * once, as a wait that ran out of time does -- it records the timeout, lets
 * its copies in flight land (a wait bounded at 2 s) and leaves -- so the calls
 * made meanwhile report FFTENKF_ETIMEOUT through fftenkf_last_device_status
 * and their outputs are incomplete.  No kernel faults or hangs.  Off (0) by
 * default; set it back to 0 to compute again. */
fftenkf_status fftenkf_set_expire_first_wait(fftenkf_plan plan, int on);

/* Per-pass timing (tracing).  With profiling enabled every pass of the calls
 * on this plan is bracketed by CUDA events on the stream it runs on.
 * fftenkf_pass_times waits for those events, writes for every pass p <
 * n_passes its total device milliseconds and number of launches since the
 * last read (or enable), and resets the totals.  Passes are numbered
 * 0..fftenkf_pass_count()-1 and named by fftenkf_pass_name.  Pass 0 ("mean")
 * is retired (the anomaly rows take the first member as pivot): it keeps its
 * number so that the others keep theirs, and always reports 0 launches. */
fftenkf_status fftenkf_set_profiling(fftenkf_plan plan, int enable);
fftenkf_status fftenkf_pass_times(fftenkf_plan plan, double* total_ms, int* launches, int n_passes);
int fftenkf_pass_count(void);
const char* fftenkf_pass_name(int pass);

/* Line-FFT schedule per pass (indexed like fftenkf_pass_name; passes without
 * transforms ignore theirs): 0 = wide plan (radix-16 stages, 16 values per
 * thread; radix 8/3 with 24 values for 3*2^a lengths), 1 = narrow plan (radix-8
 * stages, 8 values per thread, twice the threads per line).  Row passes take
 * a second bit (value 2 or 3): half as many rows per tile, so that two CTAs fit
 * on one SM.  set returns EINVAL for out-of-range entries and EUNSUPPORTED if a
 * choice does not fit
 * in shared memory; the plan keeps its previous schedule then.  The schedule
 * changes speed only: every schedule computes the same analysis. */
fftenkf_status fftenkf_set_schedule(fftenkf_plan plan, const int* sched, int n);
fftenkf_status fftenkf_get_schedule(fftenkf_plan plan, int* sched, int n);

/* ---------------------------------------------------------------- coupled observed blocks
 * coupled != 0: keep the cross-covariance between observed blocks instead of
 * neglecting it (the rule of Sec. 2.2).  eq. (multi-enkf) with the stationary
 * block covariance then gives per wavenumber k the gain of block j
 *     K_j(k) = chat_{j,O}(k) (chat_{O,O}(k) + diag(rhat_O(k)))^-1,
 * chat_{a,b} = 1/(N-1) sum_k ahat_k^(a) conj(ahat_k^(b)) (eq. dii, cov-multi-spectral),
 * and u_k^(j),a = u_k^(j) + F^-1 sum_o K_{j,o} F(d_o + e_{k,o} - u_k^(o)) for every block,
 * observed ones included.  The n_obs x n_obs bracket is inverted in FP64; where it is
 * singular (rhat = 0 and det <= 1e-6 a11 a22) its rank-1 pseudo-inverse A / tr(A)^2 is
 * used, and 0 where tr(A) = 0.  This generalises the paper, which derives the single
 * observed block.
 * Supported for one or two observed blocks when the column statistics (n_obs autos,
 * the observed pair and the n_obs x n_unobserved crosses) fit in shared memory; EUNSUPPORTED
 * otherwise (the plan keeps its mode).  The workspace grows (gains of every block);
 * a plan-owned workspace is reallocated on the next call, a caller workspace must be
 * resized from fftenkf_workspace_size.  With coupling fftenkf_estimate_spectrum writes,
 * after the observed autos, for every observed o (ascending) chat^(jo) of every block
 * j != o (ascending), and fftenkf_analyze does not accept a caller spectrum (EUNSUPPORTED).
 * Not thread-safe against concurrent calls on the same plan. */
fftenkf_status fftenkf_set_coupled(fftenkf_plan plan, int coupled);

/* ---------------------------------------------------------------- batched
 * Many independent analyses of uneven sizes (the block-state method with one
 * fully observed block each, H = I, eq. spectral-enkf), replayed as one CUDA
 * graph (captured on the first call, after every autotune, and when the
 * pointers of an analysis of at least 512 x 256 points change).  Analyses of at
 * least 512 x 256 grid points run through the single-analysis passes (one plan
 * each, created with the batch), issued on eight graph branches, largest first,
 * each to the branch with the least work; every other analysis goes through
 * seven persistent launches, each over a work list mixing the units of all of
 * them, on a branch of its own.  dims[i].n_blocks must be 1; all analyses
 * share one storage type; ny and nx/2 in {2^a, 3*2^a} between 16 and 1024.
 * The pointer arguments of fftenkf_analyze_batched are HOST arrays of `count`
 * DEVICE pointers with the single-analysis layouts (ensemble [N][ny][nx],
 * data [ny][nx] float, perturbations [N][ny][nx], rhat [ny][nx/2+1] double). */
typedef struct fftenkf_batch_s* fftenkf_batch;
fftenkf_status fftenkf_plan_batched(fftenkf_batch* batch, int count, const fftenkf_dims* dims);
fftenkf_status fftenkf_batch_destroy(fftenkf_batch batch);
fftenkf_status fftenkf_batch_workspace_size(fftenkf_batch batch, size_t* bytes);
fftenkf_status fftenkf_analyze_batched(fftenkf_batch batch, void* const* ensembles, const float* const* data,
                                       const void* const* perturbations, const double* const* rhat,
                                       void* workspace, void* stream);
/* Autotuner: times every candidate CTA size (128, 256 threads) and line-FFT
 * schedule (0, 1) of every pass on zero-filled scratch inputs of the batch's
 * shapes (allocated for the call: one copy of every item's inputs) and keeps
 * the fastest; best_ms (may be NULL) receives the sum of the best pass times. */
fftenkf_status fftenkf_batch_autotune(fftenkf_batch batch, void* workspace, void* stream, double* best_ms);
/* Chosen CTA size and schedule of each batched pass (7 passes: mean, anomaly
 * rows, statistics, gain, innovation rows, update, inverse rows). */
fftenkf_status fftenkf_batch_schedule(fftenkf_batch batch, int* cta_threads, int* sched, int n);
fftenkf_status fftenkf_batch_last_device_status(fftenkf_batch batch, void* stream);

/* ---------------------------------------------------------------- learned spectrum
 * A spectral-variance denoiser (not part of the paper's method, which only
 * motivates estimating the covariance from a very small ensemble, Sec. 2.1):
 * the single-table chat of eq. (dii) is reduced to 128 radial bins of log chat
 * (|k| = sqrt(k_y^2 + k_x^2), bin width sqrt(ny^2+nx^2)/256, bin decisions in
 * FP64), a 256 -> 64 -> 64 -> 64 -> 128 GELU MLP (BF16 weights, FP32
 * accumulation) maps the bin values minus their mean plus log bin centres to
 * the binned log spectrum of a large ensemble, and the result is interpolated
 * back to every wavenumber.  Parameters: one flat float vector of
 * fftenkf_mlp_param_count() values [W1 (64x256, row = output), b1, W2 (64x64),
 * b2, W3, b3, W4 (128x64), b4]; forward and backward use their BF16 rounding.
 * All array arguments are device pointers; spectra are [ny][nx/2+1] double.
 * A denoiser holds device scratch that fftenkf_denoiser_features and fftenkf_denoise_spectrum
 * write: calls on one denoiser must be ordered (one stream, or synchronised between streams);
 * separate denoisers run concurrently. */
typedef struct fftenkf_denoiser_s* fftenkf_denoiser;
int fftenkf_mlp_param_count(void);
fftenkf_status fftenkf_denoiser_create(fftenkf_denoiser* d, int ny, int nx, int trained_members);
fftenkf_status fftenkf_denoiser_destroy(fftenkf_denoiser d);
/* features [batch][256] float and removed means [batch] of `batch` consecutive chat tables */
fftenkf_status fftenkf_denoiser_features(fftenkf_denoiser d, const double* chat, int batch, float* features,
                                         float* means, void* stream);
/* network outputs [batch][128] (binned log spectrum minus the input mean) */
fftenkf_status fftenkf_mlp_forward(const float* params, const float* features, int batch, float* out, void* stream);
/* gradient of mean((out - targets)^2) over batch x 128 into grads (overwritten), loss into *loss (device) */
fftenkf_status fftenkf_mlp_gradient(const float* params, const float* features, const float* targets, int batch,
                                    float* grads, float* loss, void* stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step counts from 1) */
fftenkf_status fftenkf_mlp_adam(float* params, float* m, float* v, const float* grads, int step, float lr,
                                void* stream);
/* chat_out = learned spectrum of chat_in; the plain chat_in is copied instead when n_members differs
 * from the trained ensemble size or the network output is not finite.  used_fallback (HOST, may be
 * NULL; non-NULL makes the call wait for the stream) receives 1 when the plain estimate was used. */
fftenkf_status fftenkf_denoise_spectrum(fftenkf_denoiser d, const float* params, const double* chat_in,
                                        double* chat_out, int n_members, int* used_fallback, void* stream);

/* ---------------------------------------------------------------- real sine transform
 * The variant of Sec. 4: the real sine FFT in place of the periodic DFT, which leaves the
 * boundary unchanged.  The grid ny x nx includes its boundary nodes (first and last row and
 * column); the (ny-2) x (nx-2) interior is transformed by the orthonormal type-I sine transform
 * S_m[k][j] = sqrt(2/(m+1)) sin(pi (k+1)(j+1)/(m+1)) in each direction, and eq. (dii) and
 * eq. (spectral-multi-enkf) are applied with S in place of F (real coefficients; observed
 * blocks' mutual cross-covariances neglected as for the periodic plan; gain 0 where
 * chat + rhat == 0).  Boundary nodes of the ensemble are left as they are.
 * The transform is computed exactly as the periodic one of the odd extension of the interior to
 * the period 2(ny-1) x 2(nx-1), whose DFT is -S of the interior at the wavenumbers 1..m of each
 * axis (and their negatives) and zero on the lines 0 and m+1: the plan extends the inputs into
 * plan-owned buffers, runs the periodic analysis there and copies the interior back.  So
 * 2(ny-1) and 2(nx-1) must satisfy the periodic plan's rules (ny-1 in {2^a, 3*2^a} up to 2048,
 * nx-1 in {2^a, 3*2^a} up to 4096, both at least 8), else EUNSUPPORTED; the plan allocates
 * about 4x the ensemble, perturbations and data, and 4x the work of a periodic analysis on
 * ny x nx.  Device pointers need only the alignment of their element type.
 *   ensemble      [M][N][ny][nx] storage dtype, in place
 *   data          [n_obs][ny][nx] float; perturbations [N][n_obs][ny][nx] storage dtype
 *                 (only their interior nodes enter)
 *   rhat          [n_obs][ny-2][nx-2] double: data-error variance per sine wavenumber
 *                 (R = r I on the interior gives rhat = r)
 *   spectrum_out  fftenkf_sine_spectrum_size doubles: n_obs auto tables chat^(oo) followed by
 *                 n_obs * n_unobserved cross tables chat^(jo) (observed o ascending, then
 *                 unobserved j ascending), each [ny-2][nx-2] real. */
typedef struct fftenkf_sine_plan_s* fftenkf_sine_plan;
fftenkf_status fftenkf_sine_plan_create(fftenkf_sine_plan* plan, const fftenkf_dims* dims,
                                        const uint8_t* observed_mask);
fftenkf_status fftenkf_sine_plan_destroy(fftenkf_sine_plan plan);
fftenkf_status fftenkf_sine_spectrum_size(fftenkf_sine_plan plan, size_t* n_doubles);
fftenkf_status fftenkf_sine_estimate_spectrum(fftenkf_sine_plan plan, const void* ensemble, double* spectrum_out,
                                              void* stream);
fftenkf_status fftenkf_sine_analyze(fftenkf_sine_plan plan, void* ensemble, const float* data,
                                    const void* perturbations, const double* rhat, void* stream);
fftenkf_status fftenkf_sine_last_device_status(fftenkf_sine_plan plan, void* stream);

/* Morphing transform around the analysis (Sec. 2.2, eq. morphing-transform and eq. inverse-morphing).
 * The registration mappings T_k (displacement fields in grid units, T_x along x then T_y along y)
 * are the caller's.  On the periodic ny x nx grid, f o (I + T) at node p is f(p + T(p)), f
 * interpolated bilinearly between nodes; (I + T)^-1(p) is the fixed point q = p - T(q), reached by
 * at most n_iter (0..1024) steps from q = p, which converges when T is a contraction (max |grad T|
 * < 1); a node stops after the first step that moves it by at most tol cells in each component
 * (tol = 0: only when an iterate repeats exactly, the result of all n_iter steps).
 * FP32 device arrays, 4-byte aligned, row-major with x fastest:
 *   u       [M][K][ny][nx] physical members (the analysis layout with N = K)
 *   u_ref   [M][ny][nx] the reference member u_{N+1}
 *   ext     [M+2][K][ny][nx] extended ensemble (T_x, T_y, r^(1), ..., r^(M)): an FP32 analysis
 *           ensemble with n_blocks = M+2 whose observed blocks are 0, 1, 2.
 * fftenkf_morph_forward reads T from ext blocks 0, 1 and writes r_k^(j) = u_k^(j) o (I+T_k)^-1 -
 * u_ref^(j) into blocks 2..M+1 (eq. morphing-transform).  The data maps the same way with M = K = 1:
 * u = d, u_ref = the first block of the reference, ext = the [3][ny][nx] data of the analysis.
 * fftenkf_morph_reference writes the member mean of ext [C][K][ny][nx] to ext_ref [C][ny][nx]: the
 * transformed reference member after the analysis.
 * fftenkf_morph_inverse writes u_out[j][k] = (u_ref^(j) + r_k^(j)) o (I + T_k) (eq.
 * inverse-morphing); with K = 1 and ext = the reference mean it gives the new reference member.
 * Outputs must not overlap inputs (EINVAL).  Displacements are taken modulo the grid (offsets beyond
 * 2^22 cells are clamped for indexing); a non-finite displacement gives non-finite outputs, never an
 * out-of-grid read.  Errors: EINVAL (null, misaligned or overlapping pointers, dims < 1, n_iter out
 * of range, tol negative or not finite), EUNSUPPORTED (ny * nx > 2^31 - 2^20, n_members > 65535), ECUDA (launch
 * failed).  Asynchronous on stream. */
fftenkf_status fftenkf_morph_forward(const float* u, const float* u_ref, float* ext, int n_blocks, int n_members,
                                     int ny, int nx, int n_iter, float tol, void* stream);
fftenkf_status fftenkf_morph_reference(const float* ext, float* ext_ref, int n_channels, int n_members, int ny,
                                       int nx, void* stream);
fftenkf_status fftenkf_morph_inverse(const float* ext, const float* u_ref, float* u_out, int n_blocks,
                                     int n_members, int ny, int nx, void* stream);

/* Static description of a status code. */
const char* fftenkf_status_string(fftenkf_status s);
/* Message of the last failing call on this host thread ("" if none). */
const char* fftenkf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FFTENKF_H */
