/*
 * pmace.h -- C ABI of the GB300 PMACE hot path.
 *
 * PMACE (Projected Multi-Agent Consensus Equilibrium, Zhai, Buzzard,
 * Wohlberg, Bouman, arXiv 2111.14240) reconstructs a complex transmittance
 * image x (N1 x N2) from far-field amplitudes y_j (Np x Np) measured at J
 * probe positions, with a known complex probe d (Np x Np) (Section II,
 * forward model z_j = Pois(|F D P_j x|^2), y_j = sqrt(z_j)).  One iteration
 * of Algorithm 1 applies the J probe-weighted proximal agents F_j (Section
 * III-A, equation F-interpolate), the probe-weighted consensus G (equation
 * xjbar) and the Mann step v <- v + 2 rho (z - w).
 *
 * Conventions shared by every call:
 *  - complex arrays are interleaved float32 (re, im), row-major, C order;
 *  - F is the 2-D orthonormal DFT with the DC term at index [0][0] and no
 *    fftshift, so y_j must be given in that layout;
 *  - a `stream` argument is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream); calls are asynchronous on it unless stated;
 *  - the library copies every input it keeps; callers keep ownership of
 *    their buffers and may free them once the call has returned (host
 *    buffers) or once the stream has passed the call (device buffers);
 *  - no call aborts the process; every failure is reported as a status and
 *    the message is available from pmace_last_error().  A status other than
 *    PMACE_OK leaves the handle valid unless documented otherwise.
 *  - the library runs on the CUDA device that is current when pmace_create
 *    is called; later calls on the handle must be made with that device
 *    current;
 *  - calls on one handle must follow one another on the GPU (one stream, or
 *    streams the caller synchronises): they share the job's stacks and the
 *    consensus gather's scratch partial sums and tile counters.
 */
#ifndef PMACE_H
#define PMACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmace_job* pmace_handle;

typedef enum {
    PMACE_OK = 0,
    PMACE_ERR_INVALID_ARG = 1,      /* bad pointer, size, offset or amplitude value */
    PMACE_ERR_OOM = 2,              /* device or host allocation failed */
    PMACE_ERR_CUDA = 3,             /* a CUDA runtime call failed */
    PMACE_ERR_UNSUPPORTED_SIZE = 4, /* Np not in {32, 64, 128, 256} */
    PMACE_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up */
    PMACE_ERR_STATE = 6             /* call not valid in the handle's current state */
} pmace_status;

typedef enum {
    PMACE_AMP_F32 = 0,        /* amps: float32 [J][Np][Np] */
    PMACE_AMP_F16_SCALED = 1  /* amps: IEEE binary16 codes [J][Np][Np]; y = code * scales[j] */
} pmace_amp_format;

/* Problem sizes (Section II): image N1 x N2 (n1 rows, n2 columns), probe and
 * detector Np x Np, J probe positions; kappa is the probe exponent of the
 * consensus weights |D|^kappa (equation xjbar); it is fixed at creation
 * because the weight image Lambda = sum_j P_j^t |D|^kappa depends on it. */
typedef struct {
    int32_t n1, n2, np, J;
    float kappa;
} pmace_dims;

/* Per-call iteration parameters: alpha >= 0 is the noise-to-signal ratio of
 * the agents (equation F-interpolate), rho in (0, 1) the Mann averaging
 * parameter (Algorithm 1). */
typedef struct {
    float alpha, rho;
} pmace_step;

/* Create a reconstruction job: copies the inputs to the device, builds the
 * scan-overlap lists and the weight image Lambda, and sets Algorithm 1's
 * initial stacks w = v = [P_j x^(0)]_j.
 *   dims    : sizes and kappa; 1 <= Np <= min(n1, n2), J >= 1, kappa finite.
 *   probe   : d, Np*Np complex (2*Np*Np floats).
 *   offsets : J*2 int32, (row, col) of the top-left corner of window j; each
 *             must satisfy 0 <= row <= n1-Np and 0 <= col <= n2-Np
 *             (P_j extracts x[row:row+Np, col:col+Np]).
 *   amps    : measured amplitudes y_j in the layout of `fmt`; values must be
 *             finite and >= 0 (checked on the device; INVALID_ARG otherwise).
 *   scales  : J float32 per-pattern scales for PMACE_AMP_F16_SCALED, else NULL.
 *   init    : x^(0), n1*n2 complex, or NULL for the energy-matched constant
 *             c = sqrt(sum_j ||y_j||^2 / (J ||d||^2)).
 *   inputs_on_device : 0 = all array inputs are host pointers, 1 = probe,
 *             amps, scales and init are device pointers (offsets and dims
 *             are always host memory).
 *   out     : receives the handle (NULL on failure).
 * Synchronises `stream` once (input validation).  Returns
 * UNSUPPORTED_SIZE for Np outside {32, 64, 128, 256}. */
pmace_status pmace_create(const pmace_dims* dims, const float* probe, const int32_t* offsets,
                          const void* amps, pmace_amp_format fmt, const float* scales,
                          const float* init, int inputs_on_device, void* stream,
                          pmace_handle* out);

/* Run n >= 0 iterations of Algorithm 1 (w <- F(v); z <- G(2w - v);
 * v <- v + 2 rho (z - w)) with the given alpha, rho.  Asynchronous; two
 * kernel launches per iteration.  Runs of iterations with an unchanged rho
 * are replayed from a CUDA graph captured once per (alpha, rho) on a stream
 * the job owns (set PMACE_GRAPHS=0 in the environment before creating the
 * job to launch every kernel directly; per-kernel profiling also launches
 * directly). */
pmace_status pmace_iterate(pmace_handle h, int32_t n, const pmace_step* step, void* stream);

/* Algorithm 1's output x_hat = Lambda^-1 sum_j P_j^t |D|^kappa v_j for the
 * current v (pixels no window covers read 0).  out: n1*n2 complex, host
 * (out_on_device = 0; the call then synchronises `stream`) or device memory.
 * With a host `out` the call also reads the job's error word after the
 * copy: if a bounded device-side wait of an earlier agent sweep gave up, the
 * image is still written but the call returns PMACE_ERR_TIMEOUT (the image
 * may be wrong).  With a device `out` the call stays asynchronous and does
 * not check; pmace_residual reports the same condition. */
pmace_status pmace_get_image(pmace_handle h, float* out, int out_on_device, void* stream);

/* The current patch stack v (J*Np*Np complex), host or device memory. */
pmace_status pmace_get_patches(pmace_handle h, float* out, int out_on_device, void* stream);

/* Residuals of the last iteration (the last iteration of each pmace_iterate
 * call writes the per-window partial sums; the ones before it skip that
 * work), computed on the device in FP64 in a fixed order and returned in
 * out[0..1]:
 *   out[0] = ||z_prev - w|| / ||w||: disagreement between the previous
 *            consensus stack and the new agent outputs (zero at the
 *            Algorithm 1 fixed point; z_prev = v before the first iteration);
 *   out[1] = sum_j ||y_j - |F D v_j| ||^2 / sum_j ||y_j||^2 at the agents'
 *            inputs (the data term of equation eq1 up to 1/(2 sigma_n^2)).
 * Synchronises `stream`.  STATE if no iteration has run yet. */
pmace_status pmace_residual(pmace_handle h, double out[2], void* stream);

/* Checkpoint.  The state is the pending stack q = v - 2 rho w (J*Np*Np
 * complex), the consensus image xbar (n1*n2 complex), the iteration count
 * and the pending rho; together they determine v = q + 2 rho P xbar.  Resuming
 * from a saved state reproduces the uninterrupted run bit for bit. */
typedef struct {
    int64_t iterations;
    float rho_pending;
    int32_t reserved;
} pmace_state_info;

pmace_status pmace_get_state(pmace_handle h, float* q, float* xbar, pmace_state_info* info,
                             int on_device, void* stream);
pmace_status pmace_set_state(pmace_handle h, const float* q, const float* xbar,
                             const pmace_state_info* info, int on_device, void* stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every agent and consensus launch while enabled.  pmace_kernel_times
 * synchronises on the recorded events and returns the summed milliseconds
 * and launch counts since the last reset (any pointer may be NULL). */
pmace_status pmace_set_profiling(pmace_handle h, int enable);
pmace_status pmace_kernel_times(pmace_handle h, double* agent_ms, int64_t* agent_launches,
                                double* consensus_ms, int64_t* consensus_launches, int reset);

/* Kernel plan of this job: for the agent kernel the variant index, its
 * cluster size (CTAs per window), threads per CTA, dynamic shared memory per
 * CTA, columns per thread of the column step, whether the amplitudes are
 * staged in shared memory, how many clusters the device holds at once, how
 * the 2-D DFT is split over the cluster (exchange 0: an in-place cross-CTA
 * butterfly stage; 1: a transposing exchange of 16 x 16 blocks between the
 * Np / 16 CTAs, which then run their column transforms locally; 2: the same
 * exchange with two windows per cluster at a time in packed FP32 lanes) and
 * the windows each cluster processes; for the consensus gather the image
 * tile shape. */
typedef struct {
    int32_t cluster, threads, smem_bytes, tile_h, tile_w;
    int32_t variant, cols_per_thread, stage_y, max_clusters;
    int32_t exchange, windows_per_cluster;
} pmace_plan;
pmace_status pmace_get_plan(pmace_handle h, pmace_plan* plan);

/* Total measured energy sum_j sum_pixels y^2 (FP64, fixed summation order)
 * of J patterns of np x np amplitudes, without allocating device memory.
 * The paper has no counterpart: it is the sum pmace_create uses for the
 * energy-matched start, offered to callers that cannot allocate device
 * memory (a caller whose device memory is owned by another allocator, or
 * that must avoid the device-wide synchronisation cudaMalloc/cudaFree can
 * cause).
 *   amps   : device pointer, layout of `fmt` (FP32, or FP16 codes with
 *            device `scales`, y = code * scales[j]).
 *   out    : device pointer to one double, written asynchronously on `stream`.
 * Limit: J <= 65536.  Larger J returns PMACE_ERR_INVALID_ARG with a message
 * from pmace_last_error(NULL); nothing is launched then.
 * Scratch: the per-window partial sums live in one fixed 512 KB array in the
 * library's device image, held by every GPU that loads the library until the
 * process exits and shared by every call.  Each call overwrites the partials
 * it uses, so nothing needs clearing, but calls whose work overlaps on the
 * GPU (different streams, or other host threads) race on that array.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  No
 * device memory is allocated or freed. */
pmace_status pmace_amplitude_energy_noalloc(const void* amps, pmace_amp_format fmt,
                                            const float* scales, int32_t J, int32_t np,
                                            double* out, void* stream);

/* ---- Data simulator (the step before the hot path) ----
 * Measured amplitudes for a known object, made on the GPU (the forward model
 * of Section II, z_j = |F D P_j x|^2, with the photon scaling of Section IV):
 *   peak <= 0 : y_j = |F D P_j x| (noiseless);
 *   peak  > 0 : y_j = sqrt(Pois(I_j peak / M_j)) * sqrt(M_j / peak), with
 *               I_j = |F D P_j x|^2 and M_j its maximum over the window
 *               (y_j = 0 where M_j = 0).
 * The Poisson counts come from the counter-based generator Philox4x32-10
 * (draw n of pixel p of window j: counter (p, j, n, 0x504d4143), key (seed
 * low 32 bits, seed high 32 bits)) and are reproducible for a given seed.
 *   dims, probe, offsets : as for pmace_create (kappa unused);
 *   object  : x, n1*n2 complex;
 *   out     : J*Np*Np float32 amplitudes in the layout pmace_create takes.
 *   on_device : 1 = probe, object and out are device pointers (offsets host).
 * Allocates a J*Np*Np complex scratch stack for the call and synchronises
 * `stream`.  UNSUPPORTED_SIZE for Np outside {32, 64, 128, 256}. */
pmace_status pmace_simulate(const pmace_dims* dims, const float* probe, const int32_t* offsets,
                            const float* object, double peak, uint64_t seed, float* out, int on_device,
                            void* stream);

/* The photon scaling alone, on given intensities: intensity (J*Np*Np
 * float32, >= 0) -> out (same layout), as pmace_simulate does after the
 * forward model (peak <= 0: out = sqrt(intensity)).  Synchronises `stream`. */
pmace_status pmace_photon_noise(const float* intensity, int32_t J, int32_t np, double peak, uint64_t seed,
                                float* out, int on_device, void* stream);

/* Check of the agent sweep's forward transform, a test aid: runs one
 * iteration of Algorithm 1 exactly as pmace_iterate(h, 1, step, stream)
 * does (the job advances by one iteration and its residuals are those of
 * this iteration) and also writes, for every window j, the 2-D DFT of the
 * agent's input times the probe, A_j = F (d . v_j) (Section III-A, equation
 * F-interpolate, before the magnitude replacement), as the sweep computed
 * it: unnormalised (np times the orthonormal F of Section II), in natural
 * frequency order with DC at index 0.  out: J*np*np complex, device memory
 * (its contents are overwritten, also while reordering).  Only jobs on an
 * exchange plan (pmace_plan.exchange 1 or 2) support it; others return
 * PMACE_ERR_UNSUPPORTED_SIZE.  Synchronises `stream`. */
pmace_status pmace_debug_spectra(pmace_handle h, const pmace_step* step, float* out, void* stream);

/* Self-test of the bounded device-side wait of the exchange-variant agent
 * sweep: a single CTA waits on a barrier nothing completes.  Returns
 * PMACE_ERR_TIMEOUT when the wait gave up after its poll limit and reported
 * it (the designed outcome; a few seconds at most), PMACE_OK if it did not
 * (a defect), CUDA on a runtime error.  Synchronises `stream`. */
pmace_status pmace_selftest_bounded_wait(void* stream);

/* Select the kernel plan: agent variant `variant` (an index into the
 * per-probe-size variant table, see pmace_plan) and consensus tile height
 * tile_h in {8, 16, 32}.  Switching to a variant with another cluster size
 * re-lays out the stored amplitudes on the device.  Synchronises `stream`.
 * INVALID_ARG for out-of-range values, UNSUPPORTED_SIZE if the device
 * cannot run the variant. */
pmace_status pmace_set_plan(pmace_handle h, int32_t variant, int32_t tile_h, void* stream);

/* Time every runnable agent variant, then every consensus tile height, on
 * this job's own data (iters timed iterations each, after two untimed ones,
 * with `step`), keep the fastest plan and report it in *chosen (may be
 * NULL).  The job's state (stacks, consensus image, iteration count, pending
 * rho) is saved first and restored afterwards, so tuning does not advance
 * the reconstruction.  Allocates a temporary copy of the state; synchronises
 * `stream`. */
pmace_status pmace_autotune(pmace_handle h, const pmace_step* step, int32_t iters, void* stream,
                            pmace_plan* chosen);

/* ---- Serving: continuous batching of reconstruction jobs on one GPU ----
 * A server owns a worker thread (ticks), an admitter thread (job creation
 * and freeing) and two CUDA streams on the device current at creation.  Jobs are queued by pmace_server_submit (from any host thread;
 * the request's host buffers are copied, so they may be reused on return)
 * and admitted in arrival order while the device bytes of the admitted jobs
 * stay within the budget, fewer than max_active_jobs run and the admitted
 * jobs do not already fill a tick (fill_pixels).  Every tick
 * runs one iteration (Algorithm 1) for every admitted job, with the
 * windows of all jobs of one probe size and amplitude format in one agent
 * launch and the image tiles of all jobs in one consensus launch; a job that
 * has run its iterations is read out, freed and reported.  A job's result
 * is the same whether it runs alone or batched with others. */
typedef struct pmace_server* pmace_server_handle;

typedef struct {
    int64_t hbm_budget_bytes;  /* 0: 80 % of the device memory free at creation */
    int32_t max_active_jobs;   /* 0: 64 */
    int32_t tile_h;            /* consensus tile height for every job: 8, 16 or 32 (0: 16) */
    int64_t fill_pixels;       /* admit while the admitted jobs' window pixels per tick
                                  (sum of J * Np^2) stay below this; 0: 2^27 */
} pmace_server_config;

/* One job: the arguments of pmace_create (host pointers only, inputs on the
 * host), the iteration count and the step parameters. */
typedef struct {
    pmace_dims dims;
    const float* probe;
    const int32_t* offsets;
    const void* amps;
    pmace_amp_format fmt;
    const float* scales;
    const float* init;
    pmace_step step;
    int32_t iterations;
} pmace_request;

/* Outcome of a job: done = 0 while queued or running.  Times are host
 * steady-clock milliseconds (submit, admission, completion).  status is the
 * job's own status (e.g. PMACE_ERR_OOM if it can never fit the budget). */
typedef struct {
    int32_t done;
    int32_t status;
    double submit_ms, start_ms, finish_ms;
    int64_t device_bytes;
} pmace_job_result;

typedef struct {
    int64_t queued, active, completed, ticks, device_bytes, budget_bytes;
} pmace_server_counters;

pmace_status pmace_server_create(const pmace_server_config* cfg, pmace_server_handle* out);
/* Queue a job; *id identifies it in later calls.  INVALID_ARG for a
 * malformed request (sizes are checked again at admission). */
pmace_status pmace_server_submit(pmace_server_handle s, const pmace_request* req, int64_t* id);
/* Non-blocking: fills *res (res->done = 0 if not finished yet) and, for a
 * finished job, copies its image x_hat (n1*n2 complex, host) to `image`
 * when non-NULL.  Results stay available until pmace_server_release. */
pmace_status pmace_server_poll(pmace_server_handle s, int64_t id, pmace_job_result* res, float* image);
/* As poll, but waits up to timeout_ms for the job; PMACE_ERR_TIMEOUT if it
 * has not finished by then (the job keeps running). */
pmace_status pmace_server_wait(pmace_server_handle s, int64_t id, int32_t timeout_ms, pmace_job_result* res,
                               float* image);
/* Forget a finished job's result (frees its host image). */
pmace_status pmace_server_release(pmace_server_handle s, int64_t id);
pmace_status pmace_server_stats(pmace_server_handle s, pmace_server_counters* stats);
/* Stop the worker (jobs still queued or running are dropped) and free everything. */
void pmace_server_destroy(pmace_server_handle s);

/* Device bytes held by the job. */
int64_t pmace_device_bytes(pmace_handle h);

/* Release everything the job holds (NULL is a no-op).  Synchronises the
 * device work of the handle first. */
void pmace_destroy(pmace_handle h);

/* Message of the last failure on h (or of the last failed pmace_create when
 * h is NULL); never NULL, empty when there was none. */
const char* pmace_last_error(pmace_handle h);

const char* pmace_status_string(pmace_status s);

/* ABI version, bumped on any incompatible change (2: pmace_plan gained the
 * exchange and windows_per_cluster fields). */
int32_t pmace_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PMACE_H */
