/*
 * crbm.h -- C ABI of the GB300 (sm_103a) CRBM-aided Monte Carlo library.
 *
 * Method: Alcalde Puente & Eremin, "Convolutional restricted Boltzmann
 * machine aided Monte Carlo: an application to Ising and Kitaev models"
 * (arXiv:2008.05401).  Every chain repeats one proposal:
 *   g block-Gibbs steps of a convolutional RBM (Sec. II, Eqs. 12-13;
 *   App. B.1, Eqs. B1-B4), then an exact Metropolis-Hastings correction
 *   with log r = [log pi(v') - log pi(v)] + [F(v') - F(v)] (App. B.2,
 *   Eq. B5 read with the target pi and P_CRBM ~ exp(-F) as the pair of
 *   distributions), where log pi is -beta E for the 2D Ising model
 *   (Sec. III, Eq. 14) or sum_l log 2cosh(beta eps_l / 2) for the Kitaev
 *   honeycomb model in its Majorana / Z2-gauge form (Sec. IV, Eq. 16).
 *
 * Conventions shared by every call:
 *   - Every call returns a crbm_status; details of a failure are kept in the
 *     context and returned by crbm_last_error().  No call aborts the process.
 *   - Host pointers are read or written only during the call.
 *   - Device memory of a job (dev_mem) belongs to the caller (for instance a
 *     torch tensor) and must stay allocated until crbm_release().
 *   - crbm_run / crbm_run_batch are asynchronous on the given CUDA stream;
 *     the crbm_read_* calls synchronise the job's last stream first.
 *   - Lattice layout ("packed"): site n = i*L + j of the L x L lattice is bit
 *     n % 32 of uint32 word n / 32; one chain holds ceil(L*L/32) words; bits
 *     at n >= L*L are zero.  A set bit is v = 1 (Ising spin s = +1; Kitaev
 *     z-bond variable eta = +1).
 *   - Random numbers: Philox4x32-10 keyed by the 64-bit seed; the counter of
 *     every draw is (block, tag, step, chain id), chain id = chain_id_base + c.
 *     A chain's trajectory therefore depends only on (seed, chain id, state,
 *     step), never on which job, batch or slot it runs in.
 *   - Limits: 2 <= L <= 32 or L a multiple of 32 up to 256 (Ising);
 *     2 <= L <= 12 (Kitaev); 1 <= K <= 8 filters; 1 <= k <= min(7, L).
 */
#ifndef CRBM_H
#define CRBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CRBM_API __attribute__((visibility("default")))
#else
#define CRBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crbm_ctx crbm_ctx;

typedef enum {
    CRBM_OK = 0,
    CRBM_EINVAL = -1,   /* bad argument, size or id                              */
    CRBM_ENOMEM = -2,   /* job does not fit the context's HBM budget or dev_mem  */
    CRBM_ECUDA = -3,    /* a CUDA runtime call failed (message in last_error)    */
    CRBM_ETIMEOUT = -4, /* a device-side wait gave up after its iteration limit  */
    CRBM_EBUSY = -5     /* job still referenced by a live CUDA graph             */
} crbm_status;

typedef enum { CRBM_ISING = 0, CRBM_KITAEV = 1 } crbm_model_kind;

/* CRBM_FP64: every pre-activation, probability, free energy and decision in
 * FP64.  CRBM_MIXED: FP32 pre-activations (hi/lo split filters), FP32
 * sigmoid/softplus with FP64 accumulation; every Bernoulli or accept/reject
 * decision that lies within the FP32 error bound of its threshold is redone
 * with the FP64 code, so the chain takes exactly the FP64 path's decisions. */
typedef enum { CRBM_FP64 = 0, CRBM_MIXED = 1 } crbm_precision;

/* Per-chain observable sums (crbm_read_observables), CRBM_NOBS per chain:
 *   Ising : sum E, sum E^2, sum |M|, sum M^2        (E of Eq. 14, M = sum s)
 *   Kitaev: sum e, sum e^2, sum c_f, sum n_vison
 * with e(eta) = -sum_l (eps_l/2) tanh(beta eps_l/2), c_f(eta) =
 * sum_l (beta eps_l/2)^2 sech^2(beta eps_l/2) (so that <E> = <e> and
 * C = beta^2 Var(e) + <c_f>), n_vison = fraction of hexagons with flux -1.
 * One term per proposal, taken on the state after the decision. */
#define CRBM_NOBS 4

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the sum of
 * crbm_job_bytes() over live jobs (0 = no cap).  *out receives the handle.
 * Errors: CRBM_EINVAL (null out, bad device), CRBM_ECUDA. */
CRBM_API int crbm_create(crbm_ctx** out, int device, size_t hbm_budget_bytes);

/* Destroy a context and the device buffers it owns (not the jobs' dev_mem). */
CRBM_API int crbm_destroy(crbm_ctx* ctx);

/* Last error message of the context ("" if none); valid until the next call. */
CRBM_API const char* crbm_last_error(const crbm_ctx* ctx);

/* Load a CRBM (Sec. II, Eqs. 12-13): W is K*k*k FP64, row-major W[f][a][b],
 * h_bias has K entries, v_bias is the single visible bias.  The weight
 * W[f][a][b] couples hidden unit (f,i,j) to visible unit ((i+a)%L,(j+b)%L)
 * (periodic cross-correlation anchored at the top-left tap).  The values are
 * copied; the caller keeps ownership.  *model_id receives the id.
 * Errors: CRBM_EINVAL (kind, K, k out of range, null pointers). */
CRBM_API int crbm_load_model(crbm_ctx* ctx, int kind, int K, int k, const double* W,
                    double v_bias, const double* h_bias, int* model_id);

/* Load a locally connected CRBM (LCRBM) for the Kitaev model with open
 * boundaries (Sec. IV, open boundary conditions).  Reading: the lattice is
 * open along the column direction j (the y-bonds from column L-1 to column 0
 * are absent; rows stay periodic) and so are the LCRBM's windows (a column
 * past L-1 contributes nothing); the hidden units of the `edge` left columns
 * and of the `edge` right columns each have their own K kernels, all other
 * columns share the bulk kernels (the paper uses edge = 3).  W holds
 * (2 edge + 1) x K x k x k FP64 values, class-major: classes 0..edge-1 are the
 * left columns j = 0..edge-1, classes edge..2 edge-1 the right columns
 * j = L-edge..L-1, class 2 edge the bulk; then W[c][f][a][b] couples hidden
 * unit (f, i, j) of class c to visible unit ((i+a) mod L, j+b).  Hidden biases
 * (K) and the visible bias are shared.  Jobs of this model simulate the
 * open-boundary Kitaev model (vison density over the L (L-1) hexagons that do
 * not cross the cut) and run in CRBM_FP64 only.
 * Errors: CRBM_EINVAL (kind not Kitaev, edge outside [1, 6],
 * (2 edge + 1) K k 2^k > 4096), CRBM_ECUDA. */
CRBM_API int crbm_load_lcrbm(crbm_ctx* ctx, int kind, int K, int k, int edge, const double* W, double v_bias,
                             const double* h_bias, int* model_id);

/* Replace the parameters of model `model_id` (same K, k; same layout as
 * crbm_load_model), for instance after a training epoch.  Waits until the
 * device is idle, then rewrites the model's tables; its jobs use the new
 * parameters from their next launch on.  Their stored F (and the exactness
 * the tempering and exchange calls rely on) refer to the old parameters until
 * the next proposal or evaluation.  Errors: CRBM_EINVAL, CRBM_ECUDA. */
CRBM_API int crbm_update_model(crbm_ctx* ctx, int model_id, const double* W, double v_bias, const double* h_bias);

/* Bytes of caller-owned device memory one job needs: packed lattices, FP64
 * temperatures and energies, observable sums and counters (and, for the
 * Kitaev kind, the L*L single-fermion energies of each lattice), 256-byte aligned.
 * Returns 0 for arguments out of range. */
CRBM_API size_t crbm_job_bytes(int kind, int L, int n_chains, int precision);

/* Create a job of n_chains chains of side L using model `model_id`.
 *   T[n_chains]   temperature of each chain (beta = 1/T), host FP64.
 *   J             Ising: J[0] (E = -J sum s_i s_j); Kitaev: J[0..2] = (Jx, Jy, Jz).
 *   seed, chain_id_base: random stream of chain c is (seed, chain_id_base + c);
 *                 chain ids must stay below 2^32.
 *   init          0: v_ij = [u < 1/2] from the stream's init tag;
 *                 1: copy init_bits (n_chains * ceil(L*L/32) packed words, host).
 *   dev_mem       caller-owned device buffer of dev_bytes >= crbm_job_bytes().
 * Evaluates F, log pi and the observables of the initial lattices in FP64 and
 * resets the sums.  The call returns after the work is complete.
 * With an LCRBM model L must be at least 2 edge.
 * Errors: CRBM_EINVAL, CRBM_ENOMEM (dev_bytes too small or budget exceeded),
 * CRBM_ECUDA. */
CRBM_API int crbm_init_chains(crbm_ctx* ctx, int model_id, int L, int n_chains, const double* T,
                     const double* J, uint64_t seed, uint64_t chain_id_base, int init,
                     const uint32_t* init_bits, void* dev_mem, size_t dev_bytes, int* job_id);

/* Enqueue S proposals per chain on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream).  Each proposal is g Gibbs steps then the MH decision;
 * correct = 0 accepts every proposal (uncorrected Gibbs sampling, the
 * paper's Ising protocol of Sec. III).  The job's step counter advances by S.
 * Errors: CRBM_EINVAL, CRBM_ECUDA (launch failure). */
CRBM_API int crbm_run(crbm_ctx* ctx, int job_id, int64_t S, int g, int correct, int precision,
             void* cuda_stream);

/* As crbm_run for n_jobs jobs, chains of different L and temperature side
 * by side: the jobs on the tensor-core form (crbm_set_tensor_cores) share ONE
 * persistent launch whatever their sides; the other jobs share one launch
 * (Kitaev: one chain per CTA of its thread-group size when the jobs' group
 * sizes agree, else 256-thread CTAs holding several chain groups); when both
 * kinds of launch are needed they
 * fork from cuda_stream onto internal side streams and join it again, so the
 * call stays ordered on cuda_stream.  The jobs must share the model kind and
 * the filter-bank shape (K, k); their models may differ.  Each job keeps its
 * own step counter and random streams, so its result equals a crbm_run of
 * that job alone.  At most 16 jobs per call; a job may appear once. */
CRBM_API int crbm_run_batch(crbm_ctx* ctx, int n_jobs, const int* job_ids, int64_t S, int g,
                   int correct, int precision, void* cuda_stream);

/* Capture `repeats` consecutive crbm_run_batch calls of the same jobs (S
 * proposals each, same g / correct / precision) into a CUDA graph and
 * instantiate it.  The jobs' step counters live in device memory, so every
 * replay continues the chains (each replay advances every job by repeats*S
 * proposals) and the result equals the same number of direct runs.  Work
 * already enqueued on the jobs is waited for.  Jobs of a live graph cannot be
 * released (CRBM_EBUSY).  *graph_id receives the id. */
CRBM_API int crbm_graph_create(crbm_ctx* ctx, int n_jobs, const int* job_ids, int64_t S, int g, int correct,
                               int precision, int repeats, int* graph_id);

/* Replay a graph on cuda_stream (asynchronous). */
CRBM_API int crbm_graph_launch(crbm_ctx* ctx, int graph_id, void* cuda_stream);

/* Wait for the graph's jobs and free the graph. */
CRBM_API int crbm_graph_destroy(crbm_ctx* ctx, int graph_id);

/* Parallel-tempering exchange correction (App. B.2, Fig. 8b), `cycles`
 * cycles enqueued on cuda_stream.  phys_job holds the physical chains x_i
 * (target pi_i at temperature T_i; the temperature belongs to the slot i),
 * rbm_job the RBM chains y_i; both jobs must use the same model and have the
 * same L, couplings and temperatures, chain by chain.  One cycle:
 *   1. every RBM chain makes one proposal of g Gibbs steps without
 *      correction (Eq. B4); log pi_i, E and the observables of the new
 *      lattice are evaluated in FP64, F in the requested precision
 *      (CRBM_MIXED: FP32 with its certified bound, so the physical and RBM
 *      chains may hold such F values; every Bernoulli and swap decision is
 *      the FP64 path's, recomputed in FP64 when inside the bounds);
 *   2. x_i and y_i are exchanged with probability min(1, a),
 *      log a = [log pi_i(y) - log pi_i(x)] + [F(y) - F(x)] (Eq. B5 with the
 *      pair (pi_i, P_CRBM)), uniform from tag 0xFFFFFFFD of chain i of
 *      phys_job at step = the cycle counter (phys_job's step counter);
 *   3. neighbouring physical chains (i, i+1), i even on even cycles and odd
 *      on odd ones, exchange lattices with probability min(1, b),
 *      log b = log pi_i(x_{i+1}) + log pi_{i+1}(x_i) - log pi_i(x_i)
 *              - log pi_{i+1}(x_{i+1}),
 *      uniform from tag 0xFFFFFFFC of chain i; the Kitaev weight at another
 *      temperature comes from the cached spectrum of the lattice;
 *   4. every physical chain adds its observables to its sums; its accept
 *      count counts the exchanges of step 2.
 * Both step counters advance by `cycles`.  The RBM job's sums and accept
 * counts are left unchanged.  If proposals (crbm_run and the like) ran on
 * phys_job since its last evaluation (or, for CRBM_FP64, a mixed tempering
 * call left FP32 free energies), its chains are first re-evaluated in FP64
 * (synchronously).  Work enqueued earlier on either job must be ordered
 * before cuda_stream by the caller.
 * Errors: CRBM_EINVAL (mismatched jobs, g, precision, step counter past
 * 2^32), CRBM_ECUDA. */
CRBM_API int crbm_pt_run(crbm_ctx* ctx, int phys_job, int rbm_job, int64_t cycles, int g, int precision,
                         void* cuda_stream);

/* Local-update Metropolis sweeps, the paper's baseline sampler (Sec. III:
 * single spin flips for the Ising model; Sec. IV: single gauge-field flips
 * for the Kitaev model, with parallel tempering), `sweeps` sweeps of every
 * chain enqueued on cuda_stream.  One sweep at step t:
 *   Ising (L even): checkerboard order, sites with (i+j) even then odd; site
 *     (i,j) flips iff u < exp(-beta dE), dE = 2 J s_ij (sum of its 4
 *     neighbours), in FP64 (precision is ignored);
 *   Kitaev: sites n = 0..N-1 in order; eta_n flips iff
 *     log u < log pi(eta with eta_n flipped) - log pi(eta), one eigen-stage
 *     per proposal (CRBM_MIXED: the df64 stage with its certified bound and
 *     FP64 recompute, so decisions equal the FP64 path's);
 *   u of site n: word n%4 of Philox block n/4, tag 0xFFFFFFFB, step t.
 * exchange = 1 follows every sweep by the neighbour temperature exchange of
 * crbm_pt_run (step 3 there, cycle counter t; Kitaev sweeps then use the
 * FP64 stage).  After each sweep (and exchange) the observables of the
 * lattice are added to the sums; the accept count counts accepted flips; F
 * and log pi of the final lattices are FP64.  The step counter advances by
 * `sweeps`.  If proposals ran on the job since its last evaluation and
 * exchange = 1, the chains are first re-evaluated in FP64 (synchronously).
 * Errors: CRBM_EINVAL (odd Ising L, bad arguments, step counter past 2^32),
 * CRBM_ECUDA. */
CRBM_API int crbm_local_run(crbm_ctx* ctx, int job_id, int64_t sweeps, int exchange, int precision,
                            void* cuda_stream);

/* Record E_phys of every chain after each later step t of the job (proposal,
 * sweep or tempering cycle; after the exchanges) into dev_trace, a
 * caller-owned device array of capacity_steps * n_chains FP64 values,
 * time-major: row t - t0 (t0 = the job's step counter at this call), column
 * = chain.  Steps past the capacity are not recorded.  dev_trace = NULL stops
 * recording.  The buffer must stay allocated while recording; CUDA graphs
 * keep the setting they were captured with.  No counterpart in the paper:
 * the input of crbm_autocorr.  Errors: CRBM_EINVAL. */
CRBM_API int crbm_set_trace(crbm_ctx* ctx, int job_id, double* dev_trace, int64_t capacity_steps);

/* Integrated autocorrelation time of each of n_series series stored
 * time-major in device memory (dev_series[t * n_series + j], t < length),
 * for the paper's comparison of samplers by the autocorrelation of the
 * energy (Sec. III, Sec. IV).  Windowed estimator with Sokal's automatic
 * window: m = mean, G(t) = (1/n) sum_{s<n-t} (x_s - m)(x_{s+t} - m),
 * tau(W) = 1/2 + sum_{t=1..W} G(t)/G(0), W = first W >= 1 with W >= c tau(W)
 * (W <= length-1; a constant series gives tau = 1/2, W = 0).  tau[n_series]
 * (FP64) and window[n_series] (int64) are host arrays.  Runs on cuda_stream
 * after the work already there, allocates its small result buffers on it
 * (stream-ordered) and returns when the results are on the host.
 * Errors: CRBM_EINVAL (null pointers, c <= 0), CRBM_ECUDA. */
CRBM_API int crbm_autocorr(crbm_ctx* ctx, const double* dev_series, int n_series, int64_t length, double c,
                           double* tau, int64_t* window, void* cuda_stream);

/* Largest n_series crbm_autocorr_noalloc accepts. */
#define CRBM_AUTOCORR_NOALLOC_MAX_SERIES 16384

/* crbm_autocorr without any device allocation, for callers that must not
 * allocate device memory during the call (a serving loop that has handed its
 * whole HBM budget to jobs, where an allocation could fail or make the
 * allocator trim).  The paper has no counterpart: same estimator and results
 * as crbm_autocorr, but the per-series results pass through a fixed device
 * array of CRBM_AUTOCORR_NOALLOC_MAX_SERIES x 16 bytes (256 KiB) in the
 * library, shared by every call on a device.  Nothing in that array has to
 * start at zero: each call's kernel writes every entry it copies back.
 * The first call on a device looks the array up (cudaGetSymbolAddress) and
 * must not happen while a stream capture is in progress on that device.
 * Calls on one device must not overlap in time (two host threads, or a call
 * on one stream while another is still running): they would race on the
 * array.  Returns when tau and window are on the host.
 * Errors: CRBM_EINVAL (n_series > CRBM_AUTOCORR_NOALLOC_MAX_SERIES, null
 * pointers, c <= 0), CRBM_ECUDA. */
CRBM_API int crbm_autocorr_noalloc(crbm_ctx* ctx, const double* dev_series, int n_series, int64_t length,
                                   double c, double* tau, int64_t* window, void* cuda_stream);

/* One training problem of crbm_train_epochs: the paper trains one CRBM per
 * temperature (Sec. IV), so many problems run side by side.  All pointers
 * are device memory owned by the caller. */
typedef struct {
    int K, k;                 /* filter bank shape: 1 <= K <= 8, 1 <= k <= min(7, L) */
    int L;                    /* lattice side of the samples, 2 <= L <= 32 */
    int n_samples;            /* samples of the epoch */
    const uint32_t* samples;  /* [n_samples][ceil(L*L/32)] packed lattices (layout of crbm_init_chains) */
    const double* targets;    /* [n_samples] t_i = beta E_phys(x_i) (Kitaev: -log pi(x_i)) */
    const int32_t* order;     /* [n_samples] visiting order of the epoch (indices into samples) */
    double* theta;            /* [K*k*k + 1 + K] parameters [W (row-major W[f][a][b]), v_bias, h_bias]; updated */
    double* adam_m;           /* [K*k*k + 1 + K] ADAM first moments; updated */
    double* adam_v;           /* [K*k*k + 1 + K] ADAM second moments; updated */
    int64_t* adam_t;          /* [1] ADAM steps taken so far; updated */
    double* losses;           /* [ceil(n_samples / batch)] loss of each minibatch, or NULL */
} crbm_train_problem;

/* Largest number of problems one kernel launch of crbm_train_epochs takes
 * (more are split over several launches). */
#define CRBM_TRAIN_MAX_PROBLEMS 64

/* One epoch of the paper's trainer (Sec. II, App. A, Algorithm 1) for each
 * of n_problems problems (host array of descriptors), enqueued on
 * cuda_stream.  The epoch visits order[0..n_samples-1] in consecutive
 * minibatches of `batch` samples (the last one holds the remainder); per
 * minibatch, in FP64:
 *   diff_i = t_i - F(x_i) (F of Eq. 13), C = mean_i diff_i,
 *   loss = mean_i (diff_i - C)^2,
 *   g = d loss / d theta = -(2/M) sum_i (diff_i - C) dF(x_i)/d theta,
 * then one ADAM step (Kingma & Ba): m <- b1 m + (1-b1) g,
 * v <- b2 v + (1-b2) g^2, t <- t+1,
 * theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * The paper uses lr = 1e-3 and batch 20 (App. D); b1 = 0.9, b2 = 0.999,
 * eps = 1e-8 are ADAM's published defaults (the paper names none).
 * Errors: CRBM_EINVAL (shapes out of range, null pointers, batch outside
 * [1, 64]), CRBM_ECUDA. */
CRBM_API int crbm_train_epochs(crbm_ctx* ctx, int n_problems, const crbm_train_problem* problems, int batch,
                               double lr, double b1, double b2, double eps, void* cuda_stream);

/* Measure the device's FMA throughput: *fp32_tflops and *fp64_tflops (2
 * flops per fused multiply-add) from a kernel of independent FMA chains on
 * every SM, timed with CUDA events (the call allocates and frees a small
 * device buffer and returns when done).  No counterpart in the paper: the
 * peaks the rooflines of the FP32 (Ising) and FP64 (Kitaev eigen-stage,
 * trainer) kernels are reported against.  Errors: CRBM_EINVAL, CRBM_ECUDA. */
CRBM_API int crbm_probe_peaks(crbm_ctx* ctx, double* fp32_tflops, double* fp64_tflops);

/* Autotune the tile shape (chains per 256-thread CTA) of model `model_id` at
 * lattice side L and `precision`: every admissible value is timed on a
 * temporary job that fills the GPU (device memory allocated and freed by this
 * call), and the fastest is used by every job of this (kind, L, K, k) created
 * afterwards in this context.  For the Kitaev kind the value sets the threads
 * of each chain's group (256 / chains, at least 32), which run its
 * eigen-stage; a different group size changes the order of that stage's FP64
 * sums (last bits of log pi), not the method.  Jobs of the tensor-core form
 * (crbm_set_tensor_cores) keep their fixed tile of 128 / L chains.
 * *best_nc / *best_us_per_proposal (may be NULL) receive the choice and its
 * time per chain-proposal in microseconds. */
CRBM_API int crbm_tune(crbm_ctx* ctx, int model_id, int L, int precision, int* best_nc,
                       double* best_us_per_proposal);

/* Choose the kernel of later proposals (crbm_run, crbm_run_batch, graphs
 * created afterwards) for eligible jobs: enable = 1 (default) runs them on the
 * tensor-core form, enable = 0 on the table kernel.  Eligible: CRBM_ISING,
 * CRBM_MIXED, L = 128, 64, 32 or 16, K <= 4, k <= 5.  There the three convolutions of a
 * proposal (Eqs. B2, B3 and the pre-activations of F, Eq. 13) are tcgen05
 * MMAs on fp16 operands: 0/1 units and integer digits of the filters
 * (W = q (c2 2^22 + c1 2^11 + c0)), whose sums are exact in FP32; the chain
 * and every decision are the same as the table kernel's and the FP64 path's,
 * the FP32 free energy carries its own certified bound, and the Bernoulli
 * redo counts differ.  Has no effect when the device lacks the shared memory.
 * Errors: CRBM_EINVAL. */
CRBM_API int crbm_set_tensor_cores(crbm_ctx* ctx, int enable);

/* Wait for the job's last enqueued work and check the context's device error
 * flag.  A raised flag is reported once and then cleared, so the context
 * stays usable; the results of the launches that raised it are void.
 * Errors: CRBM_ECUDA, CRBM_ETIMEOUT (a device-side wait ran out of cycles,
 * see crbm_set_wait_limit). */
CRBM_API int crbm_sync(crbm_ctx* ctx, int job_id);

/* Cycle limit of every device-side wait in later launches (default 2^28 SM
 * clock cycles, about 0.13 s at 2.07 GHz).  The tensor-core kernel's
 * warp-specialised pipeline waits on shared-memory mbarriers; a wait that runs
 * out raises the CTA's abort flag (its other waits then return at once),
 * raises the context's error flag, and the CTA drains its issued MMAs,
 * releases its tensor memory and ends, so a launch never stalls the device.
 * No counterpart in the paper (failure handling of the GPU pipeline).
 * Errors: CRBM_EINVAL (cycles outside [1000, 2^40]). */
CRBM_API int crbm_set_wait_limit(crbm_ctx* ctx, int64_t cycles);

/* Check of that bounded wait, enqueued on cuda_stream: one CTA of 32 threads
 * waits for phase 0 of a shared-memory mbarrier with the tensor-core
 * pipeline's wait routine, giving up after limit_cycles cycles.  arrive = 1:
 * one thread arrives first and the wait succeeds at once; arrive = 0: nothing
 * arrives, the wait runs out and raises the context's error flag, which the
 * next crbm_sync (of any job of the context) reports as CRBM_ETIMEOUT.  No
 * counterpart in the paper.  Errors: CRBM_EINVAL (limit_cycles outside
 * [1000, 2^40], arrive not 0 or 1), CRBM_ECUDA. */
CRBM_API int crbm_probe_wait(crbm_ctx* ctx, int64_t limit_cycles, int arrive, void* cuda_stream);

/* Copy per-chain FP64 values of the current states to host arrays of
 * n_chains entries each (any may be NULL): log pi, CRBM free energy F
 * (Eq. 13) and E_phys (Ising E, Kitaev e(eta)), always the FP64 path's
 * values.  After a CRBM_MIXED run the job holds F (and, for the Kitaev kind,
 * log pi) only within the certified bounds its decisions used; the call then
 * evaluates a copy of the job's lattices in FP64 (in a device buffer the
 * context owns and grows to the job's size) and returns those values,
 * leaving the job's own state unchanged.  Synchronises the job first.
 * Errors: CRBM_EINVAL (bad job id), CRBM_ECUDA, CRBM_ETIMEOUT (see crbm_sync). */
CRBM_API int crbm_read_energies(crbm_ctx* ctx, int job_id, double* logpi, double* F_crbm, double* E_phys);

/* Copy observable sums (n_chains * CRBM_NOBS FP64, chain-major), accepted
 * proposal counts (n_chains int64) and FP64-recompute counts (n_chains x 2
 * int64: Bernoulli draws, then MH decisions, redone with the FP64 code because
 * they fell inside the FP32 error bound; always 0 for CRBM_FP64).  Any pointer
 * may be NULL. */
CRBM_API int crbm_read_observables(crbm_ctx* ctx, int job_id, double* sums, int64_t* accepts,
                          int64_t* recomputes);

/* Copy the packed lattices (n_chains * ceil(L*L/32) words) and the job's
 * step counter (proposals made so far).  Together with the seed and chain
 * ids this is a complete checkpoint. */
CRBM_API int crbm_read_state(crbm_ctx* ctx, int job_id, uint32_t* bits, uint64_t* step);

/* crbm_read_state and the observable sums of crbm_read_observables for
 * several jobs with one synchronisation (no counterpart in the paper: a
 * batching convenience of this library).  For job i: bits[i] receives its
 * packed lattices (n_chains * ceil(L*L/32) words), steps[i] its step counter,
 * sums[i] its observable sums (n_chains * CRBM_NOBS doubles); the arrays
 * bits, steps and sums, and any bits[i] or sums[i], may be NULL (not read
 * back).  Host buffers are written during the call.  Errors: CRBM_EINVAL
 * (n_jobs outside 0..16, a bad job id), CRBM_ETIMEOUT as crbm_sync,
 * CRBM_ECUDA. */
CRBM_API int crbm_read_states(crbm_ctx* ctx, int n_jobs, const int* job_ids, uint32_t* const* bits,
                              uint64_t* steps, double* const* sums);

/* Restore a checkpoint (or upload new lattices): overwrite the lattices and
 * the step counter, then re-evaluate log pi and the observables in FP64 and
 * F in `precision` (CRBM_MIXED: the FP32 value with its certified bound, as
 * a mixed proposal leaves it; the sums are kept).  A resumed chain continues
 * bit-identically to an uninterrupted one: every decision is the FP64 path's
 * either way.  Errors: CRBM_EINVAL (null bits, step >= 2^32, precision). */
CRBM_API int crbm_write_state(crbm_ctx* ctx, int job_id, const uint32_t* bits, uint64_t step, int precision);

/* crbm_write_state for several jobs at once (no counterpart in the paper: a
 * batching convenience of this library).  Job i's lattices are read from
 * bits[i] (host memory, n_chains * ceil(L*L/32) words; may be NULL for an
 * empty job) and its step counter set to steps[i]; then every listed job is
 * re-evaluated as crbm_write_state does, in ONE launch (jobs of every side
 * together) followed by one synchronisation, instead of one launch and one
 * synchronisation per job.  Host buffers are read during the call only.
 * Results are identical to crbm_write_state job by job.  Errors: CRBM_EINVAL
 * (n_jobs outside 0..16, a bad or repeated job id, null pointers, a step >=
 * 2^32, bad precision), CRBM_ECUDA. */
CRBM_API int crbm_write_states(crbm_ctx* ctx, int n_jobs, const int* job_ids, const uint32_t* const* bits,
                               const uint64_t* steps, int precision);

/* Forget a job (its dev_mem may be freed afterwards) and return its bytes to
 * the context's budget. */
CRBM_API int crbm_release(crbm_ctx* ctx, int job_id);

#ifdef __cplusplus
}
#endif
#endif /* CRBM_H */
