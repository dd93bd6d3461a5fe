/*
 * mm.h -- C ABI of the GB300 messenger-field mapmaker (Huffenberger & Naess 2017,
 * "Cosmic Microwave Background Mapmaking with a Messenger Field", arXiv:1705.01893).
 *
 * Problem (Sec. 2, Eqs. 1-3): time-ordered data d = P m + n in chunks c = 0..C-1 of
 * n_c samples each; stationary noise per chunk with power spectrum N_c(f) (circulant
 * covariance, independent chunks).  The solver finds m minimising
 *     chi^2(m) = (d - P m)^T N^-1 (d - P m),
 * the minimum-variance map m = (P^T N^-1 P)^-1 P^T N^-1 d (Eq. 2), with the messenger
 * iteration of Sec. 2.1 (T = diag(tau_c), piecewise per chunk as in Sec. 4.2) or, for
 * comparison, preconditioned conjugate gradients.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Device buffers are caller-owned (e.g. torch tensors); the library never allocates
 *    or frees device memory.  All per-plan device state lives in the caller's
 *    `workspace`, sized by mm_plan_workspace_size.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless documented otherwise.
 *  - Pointing: pix int32 [n] (-1 = sample excluded), and for IQU maps cos 2psi / sin 2psi
 *    [n] in FP32 (MM_W_F32) or FP16 (MM_W_F16).  Pointing weights of a sample are
 *    (1, cos 2psi, sin 2psi) (single pencil beam, Sec. 2.1).  The plan keeps the pointing
 *    pointers: they must stay valid and unchanged for the plan's lifetime.
 *  - Maps are float64 row-major [n_pix][ncomp], ncomp = 1 (T) or 3 (I, Q, U).  Pixels that
 *    are unobserved or cut read back as 0.  Cut: a pixel is kept iff it has >= 1 hit and,
 *    for IQU, eigmin/eigmax of its 3x3 block of P^T T^-1 P is >= rcond_min.
 *  - Chunk lengths: any n_c in [4, 2^24] whose prime factors are 2, 3 and 5, with
 *    m = n_c/2 (even n_c) or n_c (odd n_c) splitting as m = M1 M2, M1 <= 512, M2 <= 4096.
 *    n_c = 2m with m a power of two in [2^8, 2^23] and a chunk offset divisible by 4 runs
 *    the compile-time kernels (and, for m = 2^21, 2^22 or 2^23 with single pointing, the
 *    fused launch), except where the plan also has general-path chunks and the chunks of
 *    that length hold at most 2^20 samples in all: those join the general batch;
 *    the other lengths run the general mixed-radix kernels.  Other lengths return
 *    MM_ERR_UNSUPPORTED.  Entry points that support only the compile-time lengths say so.
 *  - One plan, one call at a time: calls on the same plan share its workspace (buffers,
 *    counters) and must not overlap in time; order them on one stream or synchronise.
 *  - Errors: every call returns an mm_status; on failure mm_last_error() describes it.
 *    A failed call leaves caller buffers unspecified and the plan usable, except
 *    MM_ERR_STATE, which marks an entry point called out of order.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_plan_s* mm_plan;
typedef int mm_status;

enum {
  MM_OK = 0,
  MM_ERR_ARG = -1,          /* bad argument (null pointer, size, range)            */
  MM_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed         */
  MM_ERR_NOMEM = -3,        /* workspace (or state) smaller than required          */
  MM_ERR_TIMEOUT = -4,      /* a bounded device wait gave up (plain FP64 barrier;  */
                            /* fused launch under check-on-return, see below)      */
  MM_ERR_STATE = -5,        /* call out of order (e.g. iterate before set_noise)   */
  MM_ERR_SINGULAR = -6,     /* every pixel was cut                                 */
  MM_ERR_UNSUPPORTED = -7   /* valid input this version does not handle            */
};

enum { MM_W_F32 = 0, MM_W_F16 = 1 };              /* pointing weight storage           */
enum { MM_FP32_MIXED = 0 };                        /* messenger precision modes         */

/* Bytes of device workspace a plan needs.  offsets: host int64 [n_chunks+1], chunk c
 * spans samples [offsets[c], offsets[c+1]).  ncomp 1 or 3.  Pure host computation. */
mm_status mm_plan_workspace_size(int n_chunks, const int64_t* offsets, int64_t n_pix,
                                 int ncomp, int weight_dtype, size_t* bytes);

/* Create a plan over the pointing matrix P (Sec. 2, Eq. 1: one pixel block per sample).
 * Validates the chunk layout, lays out the workspace, builds FFT twiddle tables and the
 * per-pixel hit counts (int32, exact).  cos2psi / sin2psi must be NULL iff ncomp == 1.
 * workspace: device, >= mm_plan_workspace_size bytes, 256-byte aligned, caller-owned.
 * rcond_min: IQU pixel-cut threshold (Sec. 2.1 needs P^T T^-1 P invertible), e.g. 1e-3.
 * On success *out owns host memory only; release it with mm_plan_destroy. */
mm_status mm_plan_pointing(mm_plan* out, int n_chunks, const int64_t* offsets,
                           const int32_t* pix, const void* cos2psi, const void* sin2psi,
                           int weight_dtype, int64_t n_pix, int ncomp, double rcond_min,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Set the noise model and the data (Sec. 2.1 and Sec. 4.2).
 *  psd_dev:    device float64 [sum_c (n_c/2+1)]: N_c(f_k), k = 0..n_c/2 per chunk, or NULL;
 *  params:     host float64 [n_chunks][4] = (sigma, f_knee, alpha, f_sample) giving
 *              N(f) = sigma^2 (1 + (f_knee/f)^alpha), DC bin floored to bin 1; used when
 *              psd_dev is NULL (exactly one of psd_dev / params must be given);
 *  tau:        host float64 [n_chunks] messenger covariance T = diag(tau_c), or NULL for
 *              tau_c = sigma_c^2 (params) / min_k N_c(f_k) (table).  Requires N_c - tau_c
 *              >= 0 on every bin (Nbar positive semi-definite, Sec. 2.1);
 *  tod:        device float32 [n] data d.  Read during the call only.
 * Forms Nbar, d~ = rfft(d), the weight blocks P^T T^-1 P, their inverses and the pixel cut,
 * the block-Jacobi preconditioner and b = P^T N^-1 d for PCG, and lambda_max. */
mm_status mm_set_noise_psd(mm_plan p, const double* psd_dev, const double* params,
                           const double* tau, const float* tod, void* stream);

/* Host copy of lambda_max = max_c max_k Nbar_c(f_k) / tau_c, the top of the cooling
 * range (Sec. 3.1).  Synchronises `stream`. */
mm_status mm_lambda_max(mm_plan p, double* out, void* stream);

/* Run n_iter messenger iterations (Sec. 2.1), iteration i at cooling parameter
 * lambdas[i] (host array; INFINITY = the binned-map step t = d):
 *   t~ = (lambda tau_c d~ + Nbar_c (P m)~) / (lambda tau_c + Nbar_c)  per Fourier mode,
 *   m  = (P^T T^-1 P)^-1 P^T T^-1 t.
 * map_inout: device float64 [n_pix][ncomp], read as m_0, overwritten by m_{n_iter}.
 * chi2_out:  device float64 [n_iter] or NULL; chi2_out[i] = chi^2(m_i) (Eq. 3) of the map
 *            entering iteration i, summed over all Fourier modes (Sec. 3.1).
 * precision: MM_FP32_MIXED (FP32 timestreams and FFTs, FP64 pixel accumulation,
 *            3x3 solves and chi^2 sums); other values return MM_ERR_UNSUPPORTED.  The
 *            all-FP64 step is its own entry point, mm_messenger_plain_fp64, because it
 *            needs the data d itself and a work buffer that this call does not take. */
mm_status mm_messenger_iterate(mm_plan p, const double* lambdas, int n_iter, int precision,
                               double* map_inout, double* chi2_out, void* stream);

/* Fault flags of the plan's kernels since the last call, then cleared: bit 0 = a bounded
 * wait of the fused iteration kernel (one launch for the column, row and inverse column
 * passes of a batch, whose work items wait for their chunk's earlier passes) ran out after
 * about a second; the results of that iteration are then wrong.  Synchronises `stream`.
 * The solver calls (mm_messenger_iterate, mm_messenger_graph, mm_pcg_iterate,
 * mm_messenger_iterate_md, mm_messenger_adaptive) are asynchronous and, under the default
 * wait policy, do not see such an expiry: a caller that keeps the default must read these
 * flags after synchronising to know that its results are valid (or choose check-on-return,
 * below).  No counterpart in the paper: a check of this library's own scheduling. */
mm_status mm_plan_fault_flags(mm_plan p, int* flags, void* stream);

/* Wait policy of the fused iteration kernel's bounded waits.  n_polls (1 .. 2^22, default
 * 2^22, about a second): how often a waiting work item polls its chunk's counter (about
 * 256 ns apart) before it gives up, sets the plan's fault flag and carries on (its results
 * are then wrong; nothing traps or hangs).  check_on_return (0 default, 1): with 1, the
 * solver calls listed above synchronise their stream before returning and return
 * MM_ERR_TIMEOUT (flag cleared) when a wait of their own launches ran out; with 0 they stay
 * asynchronous.  A change of n_polls drops the plan's captured graphs (they are captured
 * again on next use).  Host only.  No counterpart in the paper. */
mm_status mm_plan_set_wait_policy(mm_plan p, int n_polls, int check_on_return);

/* The work list of the fused iteration kernel for a batch of `count` chunks whose complex
 * length is m1 x m2 (m1 a power of two up to 8192, m2 a multiple of the column tile width:
 * 16 up to m1 = 512, else 8192 / m1): per item (kind, chunk, index)
 * with kind 0 = column tile, 1 = row-pair job, 2 = inverse column tile, written to out
 * (int [3 * capacity]; NULL to query the count).  Host only, no GPU.  The list puts every
 * item's prerequisites (all column tiles of its chunk for a row job, all row jobs for an
 * inverse tile) before it, which keeps the kernel free of deadlock; exposed so that this
 * can be checked.  *n_items receives the number of items. */
mm_status mm_fused_item_list(int m1, int m2, int count, int* out, int capacity, int* n_items);

/* Check of the bounded wait that the fused iteration kernel's work items use: one GPU
 * thread waits for a device flag to reach 1, at most n_polls polls about 256 ns apart
 * (1 <= n_polls <= 2^22, the kernel's own limit).  flag_set != 0 sets the flag first (the
 * wait returns at once); flag_set == 0 leaves it unset, so the wait runs out.  *expired
 * receives 1 when it ran out.  Synchronises `stream`; the GPU context stays usable either
 * way.  No counterpart in the paper: a check of this library's failure handling. */
mm_status mm_check_bounded_wait(int n_polls, int flag_set, int* expired, void* stream);

/* How many of the plan's batches mm_messenger_iterate and mm_messenger_graph run as one
 * fused launch (column, row and inverse column passes together; chunks of 2^22, 2^23 or
 * 2^24 samples, single pointing); the others run the three kernels one after the other. */
mm_status mm_plan_fused_batches(mm_plan p, int* n_fused);

/* Chunks run in batches that share one four-step FFT intermediate buffer of at most 2 GB by
 * default (environment variable MM_YBUF_MB, read when the plan is made; a budget of about a
 * quarter of L2 keeps each batch's intermediate resident in L2 between passes, at the cost
 * of more launches).
 * *n_batches receives their number; batches run one after another on the caller's stream. */
mm_status mm_plan_batches(mm_plan p, int* n_batches);

/* One stage of a messenger iteration, for callers that interleave their own work (or
 * CUDA events) between the kernels of an iteration.  mm_messenger_iterate runs one LOAD,
 * then per iteration: for each batch b, FUSED(b) where the batch is fused
 * (mm_plan_fused_batches), else GATHER_FFT(b), FILTER(b), IFFT_BIN(b); then MAP.  The same
 * sequence through this entry point gives identical results, and the three separate stages
 * on a fused batch the same up to the order of the FP64 pixel additions.
 *   MM_STAGE_LOAD:       map_inout (device float64 [n_pix][ncomp]) -> internal FP32 map;
 *   MM_STAGE_GATHER_FFT: P m gathered from the internal map, packed, column DFTs (Eq. 1);
 *   MM_STAGE_FILTER:     row DFTs, per-mode messenger filter at `lambda` (>= 1 or INFINITY),
 *                        chi^2 of the input map added to *chi2_slot if non-NULL (the caller
 *                        zeroes it), inverse row DFTs (Sec. 2.1, Sec. 3.1);
 *   MM_STAGE_IFFT_BIN:   inverse column DFTs and P^T T^-1 t into FP64 accumulators;
 *   MM_STAGE_MAP:        m = (P^T T^-1 P)^-1 acc per pixel; written to map_inout if non-NULL,
 *                        and to the internal map for the next GATHER_FFT;
 *   MM_STAGE_FUSED:      GATHER_FFT, FILTER and IFFT_BIN of the batch in one launch
 *                        (MM_ERR_UNSUPPORTED for a batch that is not fused).
 * `batch` selects the batch of the per-batch stages and is ignored otherwise; a
 * batch's GATHER_FFT, FILTER and IFFT_BIN must run in that order before the next batch's
 * GATHER_FFT (they share one intermediate buffer).  Unused pointers may be NULL. */
enum { MM_STAGE_LOAD = 0, MM_STAGE_GATHER_FFT = 1, MM_STAGE_FILTER = 2, MM_STAGE_IFFT_BIN = 3,
       MM_STAGE_MAP = 4, MM_STAGE_FUSED = 5 };
mm_status mm_messenger_stage(mm_plan p, int stage, int batch, double lambda,
                             double* map_inout, double* chi2_slot, void* stream);

/* The same iterations as mm_messenger_iterate, launched as one CUDA graph per iteration:
 * the plan captures one iteration (every batch's kernels and the map step) on its first
 * call, with the cooling parameter and the chi^2 slot read from a device-side schedule
 * table and iteration counter, and replays it n_iter times (n_iter <= 65536).  `lambdas`
 * (host) is copied to the device before the call returns.  The first call does the
 * capture on a stream the plan owns, so it must not itself be made while `stream` is
 * being captured.  Results equal mm_messenger_iterate's. */
mm_status mm_messenger_graph(mm_plan p, const double* lambdas, int n_iter, double* map_inout,
                             double* chi2_out, void* stream);

/* Bytes of device work space mm_messenger_plain_fp64 needs.  The plain step takes plans
 * whose chunks all have one compile-time length (power-of-two half); others return
 * MM_ERR_UNSUPPORTED. */
mm_status mm_plain_work_bytes(mm_plan p, size_t* bytes);

/* The plain FP64 messenger iteration, the same-GPU comparison bar of the FP32 path: per
 * iteration one cooperative launch doing, all in float64, the gather of d - P m, radix-2
 * Stockham FFTs through global memory, the filter t = d - irfft(b (d - Pm)~) (b = Nbar /
 * (lambda tau + Nbar), the residual form of Sec. 2.1's update), FP64 binning and the 3x3
 * solve, with grid-wide barriers between phases.  tod: the device float32 data given to
 * mm_set_noise_psd (the plan does not keep it).  Otherwise the arguments and results of
 * mm_messenger_iterate (to FP32 rounding of that path), plus a work buffer sized by
 * mm_plain_work_bytes.  Synchronises `stream`; a barrier that does not complete within about
 * two seconds returns MM_ERR_TIMEOUT. */
mm_status mm_messenger_plain_fp64(mm_plan p, const float* tod, const double* lambdas,
                                  int n_iter, double* map_inout, double* chi2_out, void* work,
                                  size_t work_bytes, void* stream);

/* Bytes of device work space mm_messenger_adjoint needs for n_iter iterations with a
 * checkpoint every ckpt_every iterations (caller-owned, 256-byte aligned). */
mm_status mm_adjoint_work_bytes(mm_plan p, int n_iter, int ckpt_every, size_t* bytes);

/* Gradient through n_iter messenger iterations (the forward of mm_messenger_iterate from
 * map_in with the cooling sequence `lambdas`, held constant): given grad_map_out =
 * dL/dm_{n_iter} (device float64 [n_pix][ncomp]) of any scalar loss L, writes
 *   grad_tod   = dL/dd   (device float32 [n], original sample order, overwritten), and
 *   grad_theta = dL/d(sigma, f_knee, alpha) per chunk (device float64 [n_chunks][3],
 *                overwritten; NULL to skip) -- defined when the noise came from `params`
 *                with tau = sigma^2 (MM_ERR_UNSUPPORTED otherwise).
 * The transposed step of Sec. 2.1's iteration (u = W gbar, v = P u; dL/dd += irfft(a v~)/tau,
 * dL/dm = P^T irfft(b v~)/tau, with a = lambda tau / (lambda tau + Nbar), b = 1 - a) runs on
 * the GPU for every iteration in reverse; forward iterates are recomputed from checkpoints
 * taken every ckpt_every iterations (the plan's own buffers are reused).  FP32 timestreams
 * and FFTs, FP64 accumulation.  Compile-time chunk lengths only (power-of-two halves), up
 * to 2^22 samples; other plans return MM_ERR_UNSUPPORTED.  Asynchronous on `stream`. */
mm_status mm_messenger_adjoint(mm_plan p, const double* lambdas, int n_iter,
                               const double* map_in, const double* grad_map_out,
                               float* grad_tod, double* grad_theta, int ckpt_every,
                               void* work, size_t work_bytes, void* stream);

/* The two halves of mm_messenger_adjoint, for a caller (an autograd function) that runs the
 * forward itself.  mm_messenger_forward_ckpt runs n_iter iterations of mm_messenger_iterate
 * on map_inout (same results) and first copies m_0, m_E, m_2E, ... (E = ckpt_every) into
 * ckpt: device float64 [ceil(n_iter / E)][n_pix][ncomp], caller-owned.
 * mm_messenger_adjoint_ckpt then runs the backward sweep from those checkpoints, with the
 * arguments, results and work space (mm_adjoint_work_bytes) of mm_messenger_adjoint.
 * With grad_theta == NULL neither needs the forward iterates: the step is affine in (m, d)
 * with the cooling sequence held constant, so its transpose, and hence dL/dd, does not
 * depend on them; the backward then reads no checkpoint and recomputes nothing (ckpt may be
 * any non-NULL pointer), and mm_messenger_adjoint skips its forward sweep.  Same errors as
 * mm_messenger_adjoint (MM_ERR_ARG for a NULL map, checkpoint or output pointer). */
mm_status mm_messenger_forward_ckpt(mm_plan p, const double* lambdas, int n_iter,
                                    double* map_inout, int ckpt_every, double* ckpt,
                                    void* stream);
mm_status mm_messenger_adjoint_ckpt(mm_plan p, const double* lambdas, int n_iter,
                                    const double* ckpt, const double* grad_map_out,
                                    float* grad_tod, double* grad_theta, int ckpt_every,
                                    void* work, size_t work_bytes, void* stream);

/* Bytes of device state mm_pcg_iterate needs (caller-owned, 256-byte aligned). */
mm_status mm_pcg_state_bytes(mm_plan p, size_t* bytes);

/* Preconditioned conjugate gradients on P^T N^-1 P m = P^T N^-1 d, the paper's comparison
 * solver (Sec. 1, Sec. 3.1), preconditioner = inverse of the per-pixel block
 * sum_c c0_c P_c^T P_c with c0_c the diagonal of N_c^-1.  restart != 0 starts from
 * map_inout (r = b - A m); restart == 0 continues from `state`.  map_inout holds the
 * iterate.  chi2_out: device float64 [n_iter] or NULL, chi^2 of the iterate entering each
 * step, from chi^2(x) = d^T N^-1 d - x.b - x.r. */
mm_status mm_pcg_iterate(mm_plan p, int n_iter, double* map_inout, void* state, int restart,
                         double* chi2_out, void* stream);

/* chi^2(m, lambda) = (d - Pm)^T N'^-1 (d - Pm), N' = N + (lambda - 1) T (Sec. 2.1; Eq. 3
 * at lambda = 1) into *chi2_dev (device float64 scalar, overwritten). */
mm_status mm_chi2(mm_plan p, const double* map, double lambda, double* chi2_dev,
                  void* stream);

/* Composite pointing (App. B): every sample carries two pointing entries,
 * P = gain_a P_a + gain_b P_b, each of the single-entry form of mm_plan_pointing (pixel
 * index, -1 = none; IQU weights (1, cos 2psi, sin 2psi) when ncomp == 3), e.g. a
 * differencing instrument with gain_a = 1, gain_b = -1.  The messenger covariance is split
 * T_A = T_B = T/2, so the map step divides by D = P_a^T T_A^-1 P_a + P_b^T T_B^-1 P_b (gains
 * squared, 3x3 blocks per pixel, cut by rcond as for one component), and
 * mm_messenger_iterate runs App. B's compact update
 *   m' = m + D^-1 P^T (Nbar / lambda + T)^-1 (d - P m)      (lambda = inf: T^-1)
 * (the map is not reset at lambda = inf: F(inf) != 0 for two components).  Arguments as
 * for mm_plan_pointing, plus the second component and the two gains (finite, not both 0);
 * every chunk runs on the general-length kernels (lengths with prime factors 2, 3, 5 up to
 * 2^21).  Available on a composite plan: mm_set_noise_psd, mm_lambda_max,
 * mm_messenger_iterate, mm_chi2, mm_chi2_modes, mm_rfft, mm_plan_maps (weight = D^-1),
 * mm_autotune / mm_set_tune / mm_get_tune; the other iteration forms and the operators
 * return MM_ERR_UNSUPPORTED.  The workspace size comes from
 * mm_plan_workspace_size_composite. */
mm_status mm_plan_workspace_size_composite(int n_chunks, const int64_t* chunk_offsets, int64_t n_pix,
                                           int ncomp, int weight_dtype, size_t* bytes);
mm_status mm_plan_composite(mm_plan* out, int n_chunks, const int64_t* chunk_offsets,
                            const int32_t* pix_a, const void* cos_a, const void* sin_a, float gain_a,
                            const int32_t* pix_b, const void* cos_b, const void* sin_b, float gain_b,
                            int weight_dtype, int64_t n_pix, int ncomp, double rcond_min,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Map-sized form of the messenger iteration (Sec. 2.1): m' = m_d(lambda) + F(lambda) m, with
 * m_d(lambda) = W P^T T^-1 F^-1[lambda tau d~ / (lambda tau + Nbar)] formed once for every
 * distinct lambda of the schedule (one row + column pass each, in order of first use) and
 * F(lambda) m = W P^T T^-1 F^-1[Nbar (P m)~ / (lambda tau + Nbar)] applied each iteration, so
 * the iterations no longer read d~.  Same result as mm_messenger_iterate up to FP32
 * rounding.  chi2_out (device [n_iter] or NULL) receives chi^2 at lambda = 1 of each
 * iteration's input map, assembled as d^T N^-1 d - 2 m . b + sum_k w_k |(P m)~_k|^2 /
 * (n N_k) with b = P^T N^-1 d.  work: caller-owned device memory, 256-byte aligned, of at
 * least mm_messenger_md_bytes(p, number of distinct lambdas) bytes (one float64
 * [n_pix][ncomp] map per distinct lambda); MM_ERR_NOMEM if smaller.  Asynchronous on
 * `stream`. */
mm_status mm_messenger_md_bytes(mm_plan p, int n_levels, size_t* bytes);
mm_status mm_messenger_iterate_md(mm_plan p, const double* lambdas, int n_iter, double* map_inout,
                                  double* chi2_out, void* work, size_t work_bytes, void* stream);

/* Plateau-driven cooling (Sec. 3.1: at each lambda chi^2 falls to a plateau, then lambda is
 * lowered), run entirely on the device as ONE CUDA graph launch: a conditional WHILE node
 * whose body is one messenger iteration plus a one-thread controller.  The run starts with
 * one lambda = inf step from map_inout, then walks levels[0..n_levels) (finite, >= 1, not
 * increasing; the last is normally 1).  chi^2 of the map entering iteration j is known once
 * iteration j runs, so after iteration i the newest measured decrease is that of iteration
 * i-2, r = (chi2[i-2] - chi2[i-1]) / chi2[i-1]; the level advances when at least
 * min_per_level (>= 2) of its iterations have run, iteration i-2 ran at this level and
 * r < rel_tol, or when max_per_level of its iterations have run (not applied to the last
 * level).  The loop ends when the last level would advance or after max_iter iterations.
 * Outputs (device): chi2_out[max_iter] (chi^2 at lambda = 1 of each iteration's input map,
 * zero beyond the run), lambda_out[max_iter] (lambda of each iteration, zero beyond),
 * *n_done (int, iterations run), map_inout (the final map).  Asynchronous on `stream`;
 * read *n_done after synchronising.  The graph is built on first use (and again after
 * mm_set_tune / mm_autotune). */
mm_status mm_messenger_adaptive(mm_plan p, const double* levels, int n_levels, double rel_tol,
                                int min_per_level, int max_per_level, int max_iter,
                                double* map_inout, double* chi2_out, double* lambda_out,
                                int* n_done, void* stream);

/* chi^2 per Fourier mode (the online convergence diagnostic of Sec. 3.1 / Sec. 4.1):
 * modes[off_c + k] = |d~_k - (P m)~_k|^2 / (n_c N'_c(f_k)), k = 0..n_c/2 for every chunk c
 * (off_c = sum of (n_c'/2 + 1) over the chunks before c; device float64), with N' = N +
 * (lambda - 1) T.  Each value has unit mean for the true map and sum_k w_k modes[k] (w_k =
 * 1 at DC and Nyquist, 2 elsewhere) is that chunk's chi^2.  *chi2_dev (or NULL) receives the
 * total as mm_chi2 does. */
mm_status mm_chi2_modes(mm_plan p, const double* map, double lambda, double* chi2_dev,
                        double* modes, void* stream);

/* Schedule of the general path (chunk lengths that are not powers of two, run by runtime
 * mixed-radix kernels; no counterpart in the paper, which gives no implementation).
 * mm_autotune measures, on this plan's own chunks and on `stream`, the column-tile width
 * (8 or 16 columns), threads per CTA of the column (256, 512) and row (256, 512, 1024)
 * kernels and the radix order (0: radix 8 first, then 4/2, 5, 3; 1: radix 4 in place of 8;
 * 2: radices 3 and 5 first) and keeps the fastest.  It launches the column passes and the
 * row pass in PCG-operator mode only, which leave no state behind (the accumulators are
 * cleared), needs mm_set_noise_psd first, synchronises `stream`, and drops a captured
 * iteration graph (recaptured on the next mm_messenger_graph).  mm_set_tune sets a schedule
 * explicitly (MM_ERR_ARG for values outside those sets); mm_get_tune reads it (NULL
 * outputs are skipped).  Results do not depend on the schedule beyond FP32 rounding.
 * Plans with only power-of-two chunks ignore all three. */
mm_status mm_autotune(mm_plan p, void* stream);
mm_status mm_set_tune(mm_plan p, int col_nb, int col_threads, int row_threads, int radix_order,
                      void* stream);
mm_status mm_get_tune(mm_plan p, int* col_nb, int* col_threads, int* row_threads, int* radix_order);

/* Operators, for testing and for callers composing their own solvers.
 * mm_apply_pointing:   tod_out[s] = (P m)_s in FP32 (Eq. 1), cut pixels contribute 0.
 * mm_apply_pointing_T: acc_out[p][c] = sum_s P_sp,c tod[s] in FP64 over every sample with
 *                      pix >= 0 (no cut), acc_out overwritten.
 * mm_rfft:             spec_out = rfft of every chunk of tod, complex64 interleaved
 *                      [sum_c (n_c/2+1)][2], unnormalised (numpy.fft.rfft convention). */
mm_status mm_apply_pointing(mm_plan p, const double* map, float* tod_out, void* stream);
mm_status mm_apply_pointing_T(mm_plan p, const float* tod, double* acc_out, void* stream);
mm_status mm_rfft(mm_plan p, const float* tod, float* spec_out, void* stream);

/* Copy plan maps out (any pointer may be NULL): hits int32 [n_pix]; valid uint8 [n_pix];
 * weight float64 [n_pix][ncomp*ncomp] = (P^T T^-1 P)^-1 blocks (0 on cut pixels);
 * available after mm_set_noise_psd (hits after mm_plan_pointing). */
mm_status mm_plan_maps(mm_plan p, int32_t* hits, uint8_t* valid, double* weight,
                       void* stream);

/* Binned map that allocates nothing (this entry point has no counterpart in the paper; it
 * exists for callers that cannot allocate device memory -- code being captured into a CUDA
 * graph, running under an allocator that must not grow, or handed only device pointers):
 *   map_out[p] = (P^T P)_p^-1 (P^T d)_p   for pixels with >= 1 hit and, for IQU,
 *   eigmin/eigmax of (P^T P)_p >= rcond_min; 0 elsewhere.
 * pix (int32 [n], -1 or any index outside [0, n_pix) = sample ignored), cos2psi / sin2psi
 * ([n], FP32 or FP16 as weight_dtype; NULL iff ncomp == 1) and tod (float32 [n]) are
 * device inputs; map_out is device float64 [n_pix][ncomp].  No workspace: the FP64
 * accumulators sit in one fixed device array of 2^18 pixels x 9 doubles (18.9 MB) that
 * every GPU loading the library keeps until the process exits; n_pix > 262144 returns
 * MM_ERR_ARG, and so does rcond_min outside [0, 1] (or NaN).  A call outside stream capture
 * looks up that array's address on the current device; a call during capture reuses the
 * last address found on that device, so make the first call on a device before any stream
 * capture (otherwise MM_ERR_CUDA).  Each call clears the part of
 * the array it uses; all calls on a device share the one array, so calls whose kernels
 * overlap on the GPU (e.g. on two streams) race.  Asynchronous on `stream`. */
mm_status mm_binned_map_noalloc(const int32_t* pix, const void* cos2psi, const void* sin2psi,
                                int weight_dtype, const float* tod, int64_t n, int64_t n_pix,
                                int ncomp, double rcond_min, double* map_out, void* stream);

/* Release the plan's host memory (the caller frees the workspace). NULL is a no-op. */
void mm_plan_destroy(mm_plan p);

/* Message of the last failed call on this host thread ("" if none). */
const char* mm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
