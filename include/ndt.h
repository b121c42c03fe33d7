/*
 * ndt.h -- C ABI of the GB300 non-linear digital tracking library
 * (after Golovich et al., "Survey-Wide Asteroid Discovery with a
 * High-Performance Computing Enabled Non-Linear Digital Tracking
 * Framework", arXiv 2503.08854).
 *
 * The library runs the data-parallel hot path of the paper's Algorithm 1 on
 * one GPU: for every candidate orbit it propagates the orbit to each
 * exposure epoch (two-body motion about the Sun, sec. 3), applies light time
 * and the observer position, projects through the exposure's tangent-plane
 * WCS (sec. 3), gathers matched-filter planes psi, phi at the nearest pixel
 * (sec. 3, Gaussian-PSF matched filter) and accumulates the constant-flux
 * stacked statistic (sec. 3, constant flux across images), then ranks orbits
 * (Algorithm 1, FindSignificantResults).
 *
 * Conventions shared by every entry point
 *   Units        AU, days (one uniform time scale), degrees in the WCS.
 *   Frame        heliocentric ecliptic, Sun fixed at the origin.
 *   Orbits       Cartesian state at a common epoch t0, structure of arrays:
 *                states[c * n_orbits + o], c = 0..5 -> x, y, z, vx, vy, vz
 *                (AU, AU/day), FP64.
 *   Pointers     every array argument may be host memory (pageable or
 *                pinned) or device memory of the context's device; the
 *                library detects which and copies host data through
 *                context-owned device buffers.  The caller owns every
 *                argument buffer; the context owns planes, metadata and
 *                scratch.
 *   Streams      work is issued on the stream given to ndt_create; entry
 *                points that return results in host memory synchronise it.
 *   Errors       every call returns an ndt_status; ndt_last_error() gives a
 *                one-line description.  No entry point aborts the process.
 *                A device-side failure (a Kepler solve that did not converge)
 *                is counted on the device and reported as NDT_ENOCONV by the
 *                call that reads results back.
 *   Threads      a context is not thread safe; use one per host thread.
 */
#ifndef NDT_H
#define NDT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NDT_OK = 0,
  NDT_EINVAL = 1,   /* bad argument (null pointer, size, layout)          */
  NDT_ENOMEM = 2,   /* device or host allocation failed                     */
  NDT_ECUDA = 3,    /* CUDA runtime error (message in ndt_last_error)       */
  NDT_ETIMEOUT = 4, /* a bounded device wait gave up                        */
  NDT_ESTATE = 5,   /* call out of order (e.g. stack before load)           */
  NDT_ENOCONV = 6   /* some Kepler solves did not converge                  */
} ndt_status;

typedef enum {
  NDT_PLANE_F32 = 0,  /* psi, phi stored as FP32                             */
  NDT_PLANE_BF16 = 1, /* BF16 values times per-exposure FP32 scales: the
                         powers of two nearest the noise sigma of psi and
                         the interior value of phi                         */
  NDT_PLANE_F16 = 2   /* FP16 values times per-exposure FP32 scales that map
                         each plane's largest magnitude to 2^14            */
} ndt_plane_dtype;

typedef enum {
  NDT_LAUNCH_PLAIN = 0,      /* one thread per orbit over all its exposures  */
  NDT_LAUNCH_PERSISTENT = 1  /* persistent work queue of (family, orbit tile,
                                exposure tile) items                        */
} ndt_launch_mode;

/* One exposure (paper sec. 3: image header with epoch, WCS and PSF width,
   observer location at the time of the image).  112 bytes, no padding. */
typedef struct {
  double mjd;          /* epoch, days                                      */
  double obs_xyz[3];   /* observer position, heliocentric ecliptic, AU     */
  double crval[2];     /* tangent point RA, Dec (equatorial), degrees      */
  double crpix[2];     /* tangent point pixel, 0-based (FITS CRPIX - 1)    */
  double cd[4];        /* CD matrix row-major: [CD1_1 CD1_2 CD2_1 CD2_2],
                          degrees per pixel                                */
  float psf_sigma_px;  /* Gaussian PSF sigma, pixels, in (0, 4]            */
  float variance;      /* constant per-pixel noise variance, used when no
                          variance plane is given; <= 0: estimate it by the
                          iterative MAD of the image                       */
  int32_t width;       /* pixels, 1 .. 32768                               */
  int32_t height;      /* pixels, 1 .. 32768                               */
} ndt_exposure;

/* Counters of one context, for benchmarking and tests. */
typedef struct {
  int64_t kernel_launches;   /* kernels this context has launched           */
  int64_t samples;           /* (orbit, exposure) pairs of the last stack   */
  int64_t valid_samples;     /* of which in bounds                          */
  int64_t kepler_failures;   /* solves that hit the iteration limit         */
  float last_stack_ms;       /* device time of the last stack kernel        */
  float last_planes_ms;      /* device time of the last plane computation   */
  float last_topk_ms;        /* device time of the last top-k               */
  int32_t orbit_tile;        /* persistent-launch tile shape in use         */
  int32_t exp_tile;
  int32_t launch_mode;
  int32_t plane_dtype;
  int64_t offchip_skipped;   /* samples of the last stack whose step, light
                                time and projection the off-chip test
                                removed (persistent form)                   */
  int64_t block_skipped;     /* of which the block cone test removed         */
  int64_t noise_bytes_read;  /* image bytes the last noise estimate streamed
                                (ndt_noise_mad, or load_exposures estimating
                                variances)                                  */
} ndt_stats;

typedef struct ndt_ctx ndt_ctx;

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream).  *out is set to NULL
   on failure. */
ndt_status ndt_create(ndt_ctx **out, int device, void *cuda_stream);

/* Free every device buffer of the context.  NULL is accepted. */
void ndt_destroy(ndt_ctx *ctx);

/* Description of the last error of this context (never NULL).  With a NULL
   context it describes the last failed ndt_create. */
const char *ndt_last_error(const ndt_ctx *ctx);

/* Physical constants used by propagation and light time.  Defaults: GM_sun
   = k^2 with the Gaussian constant k = 0.01720209895 AU^1.5/day, c =
   173.1446326742403 AU/day, obliquity 84381.406 arcsec.  gm <= 0 selects
   force-free (straight-line) motion, c <= 0 disables light time. */
ndt_status ndt_set_constants(ndt_ctx *ctx, double gm, double c_light, double obliquity_rad);

/*
 * load_exposures: store the exposure table and compute the matched-filter
 * planes of every image (paper sec. 3: a matched filter for a Gaussian PSF,
 * its width read from each image's header):
 *   psi_j(p) = sum_k P_j(k) I_j(p+k) / V_j(p+k),
 *   phi_j(p) = sum_k P_j(k)^2 / V_j(p+k),
 * P_j the Gaussian of sigma_j truncated at R = ceil(4 sigma_j) and
 * normalised to unit sum over its (2R+1)^2 window; terms outside the image
 * are dropped.  `images[j]` is a row-major FP32 height x width image;
 * `variances` is NULL (constant variance from the table) or n_exp per-pixel
 * FP32 variance planes of the same shape.  With `variances` NULL, an
 * exposure whose table variance is <= 0 gets the iterative-MAD estimate of
 * ndt_noise_mad (variance = sigma^2).  `plane_dtype` is an ndt_plane_dtype.
 * Replaces any previous exposure set.  Returns NDT_EINVAL for n_exp < 1, a
 * null image, sigma outside (0, 4], a NaN variance, a noise estimate that
 * is not positive, a singular CD matrix or a non-finite epoch.
 */
ndt_status ndt_load_exposures(ndt_ctx *ctx, const ndt_exposure *meta, int32_t n_exp,
                              const float *const *images, const float *const *variances,
                              int32_t plane_dtype);

/*
 * stack_orbits: for every orbit o and every exposure j of its family,
 * propagate o to the epoch of j (two-body, paper sec. 3), correct for light
 * time, project through the WCS of j, and if the nearest pixel
 * (floor(x + 1/2), floor(y + 1/2)) lies inside the image add psi_j, phi_j
 * there to the orbit's sums (paper sec. 3: intersections outside the image
 * are discarded and the rest combined under a constant-flux assumption):
 *   Psi_o = sum psi,  Phi_o = sum phi,  n_o = number of valid samples,
 *   nu_o  = Psi_o / sqrt(Phi_o) if Phi_o > 0 and n_o >= min_obs, else -inf.
 * Families (CSR): family f owns orbits [fam_orbit_off[f], fam_orbit_off[f+1])
 * and tests exposures fam_exp_idx[fam_exp_off[f] .. fam_exp_off[f+1]);
 * n_fam = 0 (and null CSR arrays) means every orbit tests every exposure.
 * fam_orbit_off must start at 0, end at n_orbits and be non-decreasing;
 * exposure indices must be in [0, n_exp) and unique within a family.
 * Outputs (each n_orbits long; any may be NULL): psi_sum, phi_sum (FP32),
 * nobs (int32), snr (FP32).  The per-orbit nu always stays in the context
 * for ndt_topk_candidates.  Sums are accumulated in FP32 with compensation.
 * The propagated state is double-float (FP32 pairs, ~48 bits; see
 * ndt_set_df_state) or FP64; light time and projection are double-float,
 * which keeps pixel coordinates within ~1e-7 px of an all-FP64 evaluation
 * at 0.2 arcsec pixels.
 */
ndt_status ndt_stack_orbits(ndt_ctx *ctx, const double *states, double t0, int64_t n_orbits,
                            const int64_t *fam_orbit_off, const int64_t *fam_exp_off,
                            const int32_t *fam_exp_idx, int32_t n_fam, int32_t min_obs,
                            float *psi_sum, float *phi_sum, int32_t *nobs, float *snr);

/*
 * topk_candidates: the k orbits of the last stack with the largest nu,
 * sorted by nu descending and orbit index ascending (paper Algorithm 1,
 * FindSignificantResults).  k is clamped to the number of orbits (any k up
 * to the batch size is supported); the number written is returned in *k_out
 * (may be NULL).  idx_out (int64) and
 * snr_out (FP32) hold k entries each; either may be NULL.
 */
ndt_status ndt_topk_candidates(ndt_ctx *ctx, int64_t k, int64_t *idx_out, float *snr_out,
                               int64_t *k_out);

/*
 * predict_positions: pixel coordinates of every orbit in every loaded
 * exposure, computed by the same propagation and light-time code as
 * stack_orbits (the TAN projection of the outputs is FP64):
 * xy_out[(o * n_exp + j) * 2 + {0, 1}] = (x, y), or NaN when the exposure's
 * tangent point is 90 degrees or more away (cos c <= 0).  j follows the
 * order of the table given to load_exposures.  FP64, n_orbits * n_exp * 2.
 */
/* count_candidates: the number of orbits of the last stack whose nu is at
   least min_snr (the detection threshold of Algorithm 1,
   FindSignificantResults; NaN and -inf never count), into *count (host).
   Sized for ndt_topk_candidates with that k.  NDT_ESTATE without a stacked
   batch, NDT_EINVAL for a NaN threshold or a null count.  Synchronous. */
ndt_status ndt_count_candidates(ndt_ctx *ctx, float min_snr, int64_t *count);

ndt_status ndt_predict_positions(ndt_ctx *ctx, const double *states, double t0,
                                 int64_t n_orbits, double *xy_out);

/* Decode the stored planes of exposure j (table order) into row-major FP32
   psi_out, phi_out (height x width each; either may be NULL). */
ndt_status ndt_get_planes(ndt_ctx *ctx, int32_t j, float *psi_out, float *phi_out);

/* Select the launch form of stack_orbits: NDT_LAUNCH_PLAIN, or
   NDT_LAUNCH_PERSISTENT with orbit_tile in {32, 64, 128} and exp_tile in
   {8, 16, 32}; use_graph != 0 replays the persistent stack through a
   captured CUDA graph when the arguments repeat. */
ndt_status ndt_set_launch(ndt_ctx *ctx, int32_t mode, int32_t orbit_tile, int32_t exp_tile,
                          int32_t use_graph);

/* Filter broadening for coarse searches (paper sec. 5.2.4: smoothing the
   images with a Gaussian wider than the PSF lets orbits be sampled more
   sparsely while still gaining signal from objects on adjacent orbits).
   From the next load_exposures on, the matched filter of exposure j uses the
   Gaussian of sigma_j' = sqrt(sigma_j^2 + sigma_px^2), the PSF smoothed by a
   Gaussian of sigma_px; 0 (the default) restores the plain filter.
   sigma_px must be finite and >= 0 (else NDT_EINVAL); load_exposures returns
   NDT_EINVAL when a broadened sigma exceeds 4 px. */
ndt_status ndt_set_filter_broadening(ndt_ctx *ctx, float sigma_px);

/* Off-chip test of the persistent form (on by default; the plain form never
   uses it).  Before the two-body step of a sample, an FP32 second-order
   prediction of its pixel with a rigorous error bound (Taylor remainder from
   the orbit's perihelion jerk bound, light time, FP32 rounding, TAN stretch)
   is compared with the image; when every lane of a warp is certainly off
   the chip the warp skips the sample and the next computed step starts from
   the last computed state.  The stacked sums are those of the full
   computation (skipped samples are out of bounds); only the rounding of the
   chained state differs.  No counterpart in the paper: its Algorithm 1
   propagates every (orbit, image) pair.  enabled = 0 switches it off. */
ndt_status ndt_set_offchip_test(ndt_ctx *ctx, int32_t enabled);

/* Block cone test of the persistent form (on by default; it acts only with
   the off-chip test on).  For every staged block of exposures (the
   exp_tile records a team walks at a time, in epoch order) each warp bounds
   the sky directions its orbits can take during the block by one cone: each
   orbit's direction at the block's middle epoch, predicted in FP32 from its
   last computed state, widened by the rigorous error bound of the off-chip test,
   the motion over the block and the spread of the block's observer
   positions.  Exposures whose chip cone (tangent point, largest off-axis
   angle + 0.01 rad) lies outside the warp's cone are skipped by the whole
   warp at a few FP32 instructions each instead of one off-chip test per
   orbit and exposure: the sky index of the sparse regime, where each orbit
   meets a small fraction of many exposures (paper sec. 3: every (image,
   orbit) pair is checked by brute force there).  The stacked sums are those
   of the full computation.  enabled = 0 switches it off. */
ndt_status ndt_set_block_test(ndt_ctx *ctx, int32_t enabled);

/* All-FP64 geometry for the plain form (off by default): light time and the
   TAN projection of stack_orbits in FP64 instead of double-float (FP32
   pairs), with the nearest pixel from an FP64 floor.  Takes effect with the
   FP64 state (ndt_set_df_state(ctx, 0)).  The reference-precision variant
   the faster forms are measured against (positions agree to ~1e-7 px at 0.2
   arcsec pixels).  The persistent form always uses the double-float
   geometry. */
ndt_status ndt_set_fp64_geometry(ndt_ctx *ctx, int32_t enabled);

/* Two-body state in double-float arithmetic (on by default; enabled = 0
   selects the FP64 state): stack_orbits (both forms) and predict_positions
   carry each orbit's position, velocity and 1/|r| as FP32 pairs (~48 bits)
   through the f and g series steps (to dt^2 K <= 1e-6, one order beyond the
   FP64 series) and the universal-variable step where |alpha chi^2| <= 5e-2
   (paper sec. 3, two-body motion about the Sun); other steps convert to
   FP64, step and convert back.  On this GPU FP64 instructions retire at 1/64
   of the FP32 rate, and with an FP64 state they bound the stacking kernel.
   Positions stay within ~1e-6 px of the FP64 state's at 0.2 arcsec pixels
   over hundreds of chained steps (sqrt(n) 2^-48 |r| of rounding noise).
   With the double-float state the plain form's FP64 geometry setting is
   ignored. */
ndt_status ndt_set_df_state(ndt_ctx *ctx, int32_t enabled);

/* Footprint order (off by default): stack_orbits without families first
   orders the orbits by their sky position at the middle exposure (Morton
   interleave of the ecliptic longitude and latitude of their light-time
   corrected direction, 16 bits each, from the stack's own propagation), so
   that the orbits of a warp gather from the same image tiles and the
   off-chip and block tests can skip whole warps (the paper batches orbits
   for its GPU intersections, sec. 4.2.1; an unordered list defeats both
   tests).  Results are those of the unordered walk (each orbit's sums do
   not depend on its neighbours) and stay in the caller's order.  Costs one
   propagation per orbit and a 4-pass radix sort of n 8-byte items per call,
   with 16 n bytes of device scratch in the context.  Families given to
   stack_orbits already group orbits and are used as given. */
ndt_status ndt_set_footprint_sort(ndt_ctx *ctx, int32_t enabled);

/*
 * autotune: time the persistent stack for every orbit_tile in {32, 64, 128}
 * and exp_tile in {8, 16, 32} on the given workload (arguments as for
 * ndt_stack_orbits, without outputs), keep the fastest shape for the
 * context and write the 9 timings (ms, row-major [orbit_tile][exp_tile]) to
 * times_ms (may be NULL).
 */
ndt_status ndt_autotune(ndt_ctx *ctx, const double *states, double t0, int64_t n_orbits,
                        const int64_t *fam_orbit_off, const int64_t *fam_exp_off,
                        const int32_t *fam_exp_idx, int32_t n_fam, float *times_ms);

/*
 * Learned vetting (paper sec. 5.2.3: a network that learns to tell stacked
 * images of real detections from stacks of false ones, left there as future
 * work; the stamp and the network below are this library's reading).
 *
 * stamps: for each candidate (an index into the orbit batch `states`, SoA
 * 6 x n_orbits at epoch t0) and each loaded exposure where its predicted
 * nearest pixel is inside the image, accumulate over a 21 x 21 window centred
 * on that pixel: SPsi, SPhi, Q = sum psi^2/phi and the count n per window
 * pixel.  Channel 0 = SPsi/sqrt(SPhi) (stacked SNR, 0 where SPhi = 0);
 * channel 1 = (Q - SPsi^2/SPhi - (n-1)) / sqrt(2 (n-1)), the constant-flux
 * chi-square excess (0 where n < 2).  Layout [n_cand][2][21][21]; stamps_f32
 * (FP32) and stamps_bf16 (BF16 bit patterns, RNE) may each be NULL.
 * Candidate indices outside [0, n_orbits) give all-zero stamps.
 */
ndt_status ndt_stamps(ndt_ctx *ctx, const double *states, double t0, int64_t n_orbits,
                      const int64_t *cand_idx, int64_t n_cand, float *stamps_f32,
                      uint16_t *stamps_bf16);

/* Number of parameters of the vetting network: 52,929.  Flat FP32 layout:
   w1 [32][2][5][5], b1 [32], w2 [32][32][5][5], b2 [32], w3 [32][32][5][5],
   b3 [32], wl [32], bl [1].  The network: three 5x5 "same" cross-correlation
   layers with bias and ReLU (2->32->32->32 channels), global average pool,
   linear 32->1 giving a logit. */
int64_t ndt_cnn_param_count(void);

/* Logits of n BF16 stamps [n][2][21][21] on the tensor core: all three
   layers take BF16 weights (rounded from the FP32 params, RNE), layers 2 and
   3 BF16 activations, with FP32 accumulation; bias, pooling and the linear
   head are FP32.  NDT_ETIMEOUT if a bounded device wait gave up (logits then
   NaN). */
ndt_status ndt_cnn_forward(ndt_ctx *ctx, const float *params, const uint16_t *stamps_bf16,
                           int64_t n, float *logits);

/* Mean binary cross-entropy with logits over the n stamps (labels 0 or 1)
   and its gradient with respect to every parameter (grad: 52,929 FP32,
   overwritten).  loss_out and logits_out may be NULL. */
ndt_status ndt_cnn_loss_grad(ndt_ctx *ctx, const float *params, const uint16_t *stamps_bf16,
                             const float *labels, int64_t n, float *grad, float *loss_out,
                             float *logits_out);

/* One Adam step (Kingma & Ba 2015, bias-corrected, step >= 1) on device
   arrays params, m, v given the gradient grad (all n_params FP32, device
   memory only). */
ndt_status ndt_cnn_adam_step(ndt_ctx *ctx, float *params, const float *grad, float *m, float *v,
                             int64_t n_params, int32_t step, float lr, float beta1, float beta2,
                             float eps);

/*
 * noise_mad: per-image noise by the iterative median absolute deviation
 * (paper sec. 3: each image's pixel noise variance comes from an iterated
 * MAD of its pixels).  For image i (n_pixels[i] FP32 values at
 * images[i], host or device memory), with S_0 = every pixel:
 *   m = lower median of S (the element of rank floor((n-1)/2)),
 *   sigma = fl32(1.4826 * lower median of fl32|x - m| over S),
 *   S' = { x : fl32|x - m| <= fl32(3 sigma) } over every pixel,
 * repeated until (m, sigma) repeats or max_rounds (1..100) rounds; outputs
 * median_out[i], sigma_out[i] and rounds_out[i] (any may be NULL; host or
 * device, caller-owned).  The result is exact: FP32 operations as written
 * and exact order statistics.  An image with no pixels gives NaN; an
 * image of more than 2^32 - 1 pixels, a null image with pixels or
 * max_rounds outside 1..100 gives NDT_EINVAL.  Device memory of the
 * context: about 1 MB per image (the selection's key buffer) plus a staging
 * copy of host images.  A selection usually streams the image once or
 * twice (ndt_stats.noise_bytes_read counts the bytes).
 * load_exposures uses the same estimate (variance = sigma^2) for exposures
 * whose variance is <= 0 when no variance planes are given.  Synchronous.
 */
ndt_status ndt_noise_mad(ndt_ctx *ctx, const float *const *images, const int64_t *n_pixels,
                         int32_t n_images, int32_t max_rounds, float *median_out, float *sigma_out,
                         int32_t *rounds_out);

/*
 * trim_candidates: outlier trimming of candidates' intersections (paper
 * sec. 5.2.3 drops intersections whose SNR lies far above what the
 * candidate predicts, by sigma clipping, and recomputes the stacked SNR).
 * For each candidate cand_idx[i] (an index into the orbit batch `states`, SoA
 * 6 x n_orbits as in stack_orbits, host or device), its valid intersections
 * j (nearest pixel inside the image, phi_j > 0) are clipped by the rule
 *   a = sum_K psi / sum_K phi,  r_j = psi_j / sqrt(phi_j) - a sqrt(phi_j),
 *   K' = { j : r_j <= kappa },  repeated from K = all valid until K' == K or
 *   max_iter rounds,
 * and nu_out[i] = sum_K psi / sqrt(sum_K phi) (-inf if the sum of phi is 0
 * or |K| < min_obs), nkept_out[i] = |K| (nkept_out may be NULL).  Outputs
 * n_cand FP32 / int32 values, host or device memory, caller-owned.
 * Indices outside [0, n_orbits) give -inf and 0.  kappa > 0 (INFINITY
 * keeps every intersection), 1 <= max_iter <= 1000, min_obs >= 0; else
 * NDT_EINVAL.  Uses the planes of the last load_exposures (NDT_ESTATE if
 * none).  Synchronous.
 */
ndt_status ndt_trim_candidates(ndt_ctx *ctx, const double *states, double t0, int64_t n_orbits,
                               const int64_t *cand_idx, int64_t n_cand, float kappa, int32_t max_iter,
                               int32_t min_obs, float *nu_out, int32_t *nkept_out);

/*
 * dedup_candidates: drop near-duplicate candidates from a ranked list (no
 * counterpart in the paper, whose detections come one orbit at a time; a
 * dense search finds every object through many neighbouring orbits, and
 * this reading removes them so that the list holds one entry per track).
 * cand_idx (n_cand indices into the orbit batch `states`, SoA 6 x n_orbits at
 * t0, host or device) is taken in rank order, best first, e.g. the output of
 * ndt_topk_candidates.  n_ref reference exposures are spread evenly over the
 * epoch-sorted exposures whose epochs lie in [t_lo, t_hi] (first and last
 * of them included; every exposure when t_lo > t_hi or either is NaN, and
 * NDT_EINVAL when the window holds none): a window around the epochs where
 * the candidates are observed, in a survey far longer than that; candidate i is a
 * duplicate when some candidate ranked before it has predicted pixel
 * positions (same propagation, light time and TAN projection as the stack)
 * within radius_px of i's at every reference exposure, each in that
 * exposure's own pixel grid.  The kept indices are written in rank order to
 * keep_idx (host or device, n_cand entries of room), their number to
 * *n_keep (host).  A position is undefined where the exposure's tangent
 * point is 90 degrees or more away: such a candidate is within radius_px of
 * no other, so it is kept and removes nothing.  radius_px > 0 and
 * finite, 1 <= n_ref <= 8, 0 <= n_cand <= 2^26, else NDT_EINVAL; NDT_ESTATE
 * before load_exposures.  Synchronous.
 */
ndt_status ndt_dedup_candidates(ndt_ctx *ctx, const double *states, double t0, int64_t n_orbits,
                                const int64_t *cand_idx, int64_t n_cand, float radius_px, int32_t n_ref,
                                double t_lo, double t_hi, int64_t *keep_idx, int64_t *n_keep);

/* vet: stamps of the candidates (as ndt_stamps) scored by the network:
   scores[i] = sigmoid(logit) in [0, 1]. */
ndt_status ndt_vet(ndt_ctx *ctx, const float *params, const double *states, double t0,
                   int64_t n_orbits, const int64_t *cand_idx, int64_t n_cand, float *scores);

/* Self-test of the scoring kernel's bounded waits (no counterpart in the
   paper).  Runs the tensor-core CNN forward on one zero stamp with the MMAs
   of its first layer withheld, so the mbarrier wait for them cannot complete:
   after its iteration limit (about a second per wait; the self-test meets
   two) the kernel records the timeout,
   frees its tensor memory and returns.  Returns NDT_ETIMEOUT when that path
   works (any other status means it did not); the context stays usable. */
ndt_status ndt_selftest_wait_timeout(ndt_ctx *ctx);

/*
 * topk_noalloc: the ranking of ndt_topk_candidates (k largest values, ties to
 * the lower index, NaN ranked with -inf) for callers that cannot let a
 * library allocate device memory, for example a host framework that keeps
 * nearly all of the GPU's memory in its own pool, or a real-time loop that
 * cannot pay for cudaMalloc/cudaFree between frames.  It allocates nothing:
 * its scratch is one array of 200 KB compiled into the library, held on
 * every GPU that loads the library until the process exits.  The paper has
 * no counterpart; this is an interface convenience.
 *   snr_dev   n FP32 values in device memory (e.g. the snr output of
 *             ndt_stack_orbits).
 *   n, k      1 <= n <= 67,108,864 and 1 <= k <= 8192 (k is clamped to n);
 *             anything larger returns NDT_EINVAL.
 *   idx_out   k int64 indices, snr_out k FP32 values, device memory of the
 *             same device (either may be NULL).
 *   cuda_stream  the cudaStream_t the kernels are issued on (NULL = the
 *             legacy default stream); the call returns without waiting.
 * The first call on a device looks up the array's device address (once per
 * device, with that device made current); make that first call before any
 * stream capture begins.  Every call on a device shares the one array and the
 * next call overwrites it: calls whose kernels overlap on the GPU (different
 * streams or host threads) race and must be serialised by the caller.  Host
 * pointers return NDT_EINVAL; a CUDA error returns NDT_ECUDA.
 */
ndt_status ndt_topk_noalloc(const float *snr_dev, int64_t n, int64_t k, int64_t *idx_out,
                            float *snr_out, void *cuda_stream);

/* Measured issue rate of the FP64 pipe on `device` (no counterpart in the
   paper; the denominator of the FP64-state stacking kernel's roofline,
   which is bound by FP64 instructions).  op 0 = DFMA, 1 = DMUL, 2 = DADD: every thread of a
   full-occupancy grid runs eight independent chains of that instruction;
   *inst_per_s = thread-instructions retired per second over four launches
   (after one warm-up launch), *seconds (may be NULL) = their duration.
   Allocates and frees a small output buffer; synchronous on the legacy
   default stream.  NDT_EINVAL for a bad op or device. */
ndt_status ndt_measure_fp64_rate(int device, int32_t op, double *inst_per_s, double *seconds);

/* Copy the context's counters into *out. */
ndt_status ndt_get_stats(ndt_ctx *ctx, ndt_stats *out);

/* Wait for all work issued by the context. */
ndt_status ndt_synchronize(ndt_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* NDT_H */
