/*
 * ffb.h -- C ABI of the GB300 fast Fourier-Bessel steerable PCA library.
 *
 * Method: Zhao, Shkolnisky & Singer, "Fast Steerable Principal Component
 * Analysis" (Alg. 1 "Fast Fourier-Bessel Expansion", Alg. 2 "Steerable PCA").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are float32, row-major [n][L][L].  The first array index is the
 *   pixel coordinate i1 (x), the second is i2 (y); both run over
 *   i = -ceil((L-1)/2) .. floor((L-1)/2) (Sec. II), so array position a holds
 *   i = a - L/2 (integer division).
 * - Fourier transform sign convention: F(f)(xi) = int f(x) e^{-2 pi i x.xi}
 *   (Sec. II).  The polar samples are F(I)(xi) = sum_i I(i) e^{-2 pi i xi.i};
 *   the 1/(2R)^2 factor printed in Eq. nufft is not applied, so the map from
 *   images to coefficients is close to unitary (Fig. 3).
 * - Coefficients a_{k,q} for k = 0..k_max only (a_{-k,q} = conj a_{k,q}, Sec.
 *   II-B), stored as interleaved complex float32 [n][P][2] (re, im) with the
 *   index of (k, q) equal to offset[k] + (q-1): k ascending, q ascending.
 *   Im a_{0,q} is written as exactly 0.
 * - Pointers named d_* are DEVICE pointers owned by the caller; pointers named
 *   h_* are HOST pointers owned by the caller.  The plan owns its tables, its
 *   scratch memory and the covariance accumulator.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Compute calls are asynchronous on that stream; argument errors
 *   are returned immediately, device-side errors (non-finite input, a
 *   bounded wait that timed out, Jacobi not converged) are latched in the plan
 *   and returned by the next call that synchronises (ffb_cov_get, ffb_eig,
 *   ffb_sync).  No entry point aborts the process.
 * - A plan belongs to the CUDA device that was current when ffb_plan built
 *   it (its tables and scratch live there); every entry point that works on
 *   a plan's device memory returns FFB_ERR_ARG while another device is
 *   current.
 * - Every entry point returns an ffb_status; ffb_strerror() names it.
 */
#ifndef FFB_H
#define FFB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffb_plan_s *ffb_plan_t;

typedef enum {
    FFB_OK = 0,
    FFB_ERR_ARG = -1,            /* invalid argument (size, range, NULL)        */
    FFB_ERR_CUDA = -2,           /* a CUDA runtime call failed                  */
    FFB_ERR_OOM = -3,            /* device allocation failed                    */
    FFB_ERR_NONFINITE = -4,      /* NaN/Inf met in an input image               */
    FFB_ERR_NOT_CONVERGED = -5,  /* Jacobi sweep limit reached                  */
    FFB_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up          */
    FFB_ERR_STATE = -7,          /* call out of order (e.g. eig before cov)     */
    FFB_ERR_UNSUPPORTED = -8     /* size/precision not supported by the library */
} ffb_status;

/* Arithmetic of the two dense contractions (radial quadrature, covariance). */
typedef enum {
    FFB_FP32 = 0,     /* CUDA-core FFMA, float32                              */
    FFB_BF16 = 1,     /* tensor cores, bf16 operands, fp32 accumulation       */
    FFB_BF16X3 = 2,   /* bf16 hi/lo split, 3 products (hh + hl + lh)          */
    FFB_TF32 = 3,     /* tensor cores, tf32 operands, fp32 accumulation       */
    FFB_TF32X3 = 4    /* tf32 hi/lo split, 3 products                         */
} ffb_precision;

/* Denoising modes of ffb_denoise (Sec. V). */
typedef enum {
    FFB_DENOISE_TOPK = 0,       /* keep the K (k,l) pairs of largest eigenvalue, gain 1 */
    FFB_DENOISE_MP_WIENER = 1,  /* keep lambda > sigma2 (1+sqrt(gamma_k))^2 (Eq. compselect),
                                   gain (lambda - sigma2)/lambda                          */
    FFB_DENOISE_ALL = 2,        /* every component, gain 1 (projection onto the span)    */
    FFB_DENOISE_MP_HARD = 3     /* keep lambda > sigma2 (1+sqrt(gamma_k))^2, gain 1       */
} ffb_denoise_mode;

/* ffb_plan -- Alg. 1 steps 1-2 (precomputation), Sec. II-A and II-B.
 * Selects (k, q) by the sampling criterion R_{k,q+1} <= 2 pi c R (Eq.
 * criterion1), fixes n_xi = ceil(4cR), n_theta = ceil(16cR), computes on the
 * GPU in float64 the Bessel zeros R_{k,q}, the Gauss-Legendre rule on [0, c]
 * and the radial table B^(k)_{q,j} = N_{k,q} J_k(R_{k,q} xi_j/c) xi_j w_j of
 * Eq. a, and builds the type-2 NUFFT used for Eq. nufft (exponential-of-
 * semicircle kernel, oversampling 2, width ceil(log10(1/eps)) + 2).
 *   L in [8, 512], c in (0, 1/2], R in (0, L/2], eps in [1e-7, 1e-2],
 *   precision an ffb_precision (FFB_ERR_ARG otherwise).  2L and n_theta must
 *   factor into 2, 3, 5 (FFB_ERR_UNSUPPORTED otherwise).  Every accepted
 *   size runs every entry point of this header except where one states a
 *   tighter bound (ffb_svd; the tensor-core covariance of ffb_group_*); the
 *   largest, L = 512 with R = 256 and c = 1/2, has p_0 = 255 and n_theta =
 *   2048, for which some kernels switch to smaller shared-memory tiles.
 * On success *out owns device memory until ffb_plan_destroy.  Synchronous. */
int ffb_plan(ffb_plan_t *out, int L, double c, double R, double eps,
             int precision, void *stream);

/* ffb_interp_units -- the interpolation table that ffb_plan builds for the
 * shared-memory grid path (plan_info[10] = 1 or 2), computed on the host for
 * inspection and tests; no GPU work.  It drives the type-2 NUFFT's last step
 * (Eq. nufft, Sec. III): the polar node (xi_j, theta_l), theta_l = 2 pi l /
 * n_theta, l < n_theta/2, sits at p = N xi_j (cos, sin) in grid units; its
 * w x w window of the half grid starts at row r0 = ceil(p2 - w/2) + (w+1)/2
 * and column c0 = ceil(p1 - w/2) - m1lo (m1lo = -(w+1)/2 for half 0, the
 * nodes with cos theta >= 0, i.e. l <= n_theta/4; -N/2 - (w+1)/2 for half 1),
 * with the weights phi(f - b), f = p - ceil(p - w/2), b < w, phi(x) =
 * exp(beta (sqrt(1 - (2x/w)^2) - 1)) evaluated in float64.
 *   N in {128, 256}, w = 8 (FFB_ERR_UNSUPPORTED otherwise), beta > 0 (the
 *   plan uses 2.30 w), h_xi[n_xi] the radii on [0, c] (the plan's
 *   Gauss-Legendre nodes), n_theta even.
 * h_counts[9] (out): float4 records, blocks, blocks of half 0, blocks of
 *   half 1, units per block GU, half-grid size MH, its row pitch SLD, fields
 *   per unit record F (19), nodes per unit at most (at most 4).
 * h_rec (may be NULL: sizing call): float[4 h_counts[0]], per block F fields
 *   of GU float4 ([block][field][unit]).  A unit is up to four nodes whose
 *   window origins lie in one 2 x 2 box, read from the 9 x 9 union of their
 *   windows: field q < 9 holds the column weights of union column q, one per
 *   node slot (x, y, z, w = slots 0..3); field 9 + r those of union row r;
 *   field 18 = (bits of ru | cu << 16, the union's first row and column,
 *   bits of slot0 | slot1 << 16, bits of slot2 | slot3 << 16, 0), the slots
 *   being block-local node indices as unsigned halves, 0xFFFF for none.  A
 *   node's weights are zero outside its own window (rows r0 - ru .. + 7,
 *   columns c0 - cu .. + 7, each offset 0 or 1); an empty unit has slot0 =
 *   0xFFFF.
 * h_blk (may be NULL): int[2 h_counts[1]], per block (first node t0, node
 *   count), nodes numbered t = j nl + (l - l0) within the half (nl nodes per
 *   ring of the half, l0 its first angle); half 0's blocks come first. */
int ffb_interp_units(int N, int w, double beta, int n_xi, int n_theta, const double *h_xi,
                     int64_t *h_counts, float *h_rec, int *h_blk);

/* ffb_tile_units -- the interpolation table that ffb_plan builds for the
 * separate-kernel path (plan_info[10] = 0, w = 8), computed on the host for
 * inspection and tests; no GPU work.  Same node geometry and ES weights as
 * ffb_interp_units, but the polar nodes (xi_j, theta_l), l < n_theta/2, of
 * one image form a single set: node t = j n_theta/2 + l has its window at
 * G row r0 = ceil(p2 - w/2) + h and unwrapped column u = ceil(p1 - w/2) +
 * N/2 + h (h = (w+1)/2; column u maps to m1 = u - N/2 - h, stored mod N),
 * and belongs to the tile (r0 / TR, u / TC).  A tile's nodes form units of up
 * to four whose origins lie in one 2 x 2 box, split into blocks of at most
 * GU units.
 *   N even >= 16, w = 8 (FFB_ERR_UNSUPPORTED otherwise), beta > 0, h_xi[n_xi]
 *   the radii on [0, c], n_theta even.
 * h_counts[9] (out): blocks, entries of all node lists, fields per unit
 *   record F (19), units per block GU, tile rows TR, tile columns TC, rows RS
 *   and columns CS of a tile in shared memory, its row pitch.
 * h_rec (may be NULL: sizing call): float[4 F GU h_counts[0]], per block F
 *   fields of GU float4 laid out as in ffb_interp_units, with the union origin
 *   (ru, cu) relative to the tile's first row and column and the slots
 *   indexing the block's node list.
 * h_blk (may be NULL): int[4 h_counts[0]], per block (first G row e0 of the
 *   tile, first unwrapped column u0, first entry of its node list, node
 *   count).
 * h_nodes (may be NULL): int[h_counts[1]], the node lists (values t). */
int ffb_tile_units(int N, int w, double beta, int n_xi, int n_theta, const double *h_xi,
                   int64_t *h_counts, float *h_rec, int *h_blk, int *h_nodes);

/* Releases everything the plan owns.  NULL is accepted. */
int ffb_plan_destroy(ffb_plan_t plan);

/* Sizes of the plan, written to h_info[0..10]:
 *   0 L, 1 k_max, 2 P (= sum_{k>=0} p_k), 3 n_xi, 4 n_theta,
 *   5 N (oversampled grid), 6 kernel width w, 7 precision,
 *   8 max_k p_k, 9 images per internal chunk, 10 polar transform variant
 *   (0 separate grid / interpolation kernels, 1 grid in shared memory,
 *   2 as 1 with the two CTAs of an image in a cluster sharing the FFTs;
 *   2 is chosen when such clusters fill every SM, unless the environment
 *   variable FFB_FUSED_CLUSTER is "0" when the plan is created). */
int ffb_plan_info(ffb_plan_t plan, int *h_info);

/* p_k and offset[k] (k = 0..k_max), host arrays of k_max+1 ints. */
int ffb_plan_sizes(ffb_plan_t plan, int *h_p, int *h_offset);

/* Copies the float64 setup tables to host arrays (any may be NULL):
 * h_zeros[P] = R_{k,q}; h_xi[n_xi], h_w[n_xi] = Gauss-Legendre rule on [0,c];
 * h_B[P*n_xi] = B^(k)_{q,j} row-major (coefficient index, j). */
int ffb_plan_tables(ffb_plan_t plan, double *h_zeros, double *h_xi, double *h_w,
                    double *h_B);

/* Changes the arithmetic of the dense contractions (ffb_precision). */
int ffb_set_precision(ffb_plan_t plan, int precision);

/* ffb_set_wait_budget -- the bound, in SM clock cycles, of the waits between
 * the pipeline roles of the tensor-core kernels of this plan (the TMA
 * producer, the MMA issuer and the epilogue of the radial quadrature; the
 * tile buffers and the final accumulator of the covariance).  The paper has
 * no counterpart: the default (4e9 cycles, about 2 s) only stops a wait
 * that could otherwise spin forever.  A wait that runs out latches
 * FFB_ERR_TIMEOUT, which the next synchronising call returns (and clears);
 * the kernel then waits, with the default budget whatever this setting, for
 * the copies and MMAs it has already issued, releases its tensor memory and
 * returns, so the context stays usable; the results of that call are
 * undefined.  Meant for tests of that error path: cycles = 0 makes every
 * such wait give up at once.  cycles < 0 restores the default.  FFB_ERR_ARG
 * for a null plan. */
int ffb_set_wait_budget(ffb_plan_t plan, long long cycles);

/* ffb_polar -- Eq. nufft at the polar nodes with theta_l in [0, pi):
 * d_F[n][n_xi][n_theta/2][2] (interleaved complex, float32); the other half
 * of every ring is the complex conjugate (real images).  Exposes steps
 * a1-a3 of the path (precorrect, oversampled FFT, interpolation). */
int ffb_polar(ffb_plan_t plan, const float *d_images, int64_t n, float *d_F,
              void *stream);

/* ffb_polar_noalloc -- the same polar samples as ffb_polar, computed without
 * allocating device memory.  The paper has no counterpart: this entry point
 * exists for callers that must not call cudaMalloc on the calling path
 * (code running during CUDA stream capture, latency-bound serving loops,
 * host frameworks that own all device memory).  Scratch comes from a 16 MiB
 * array that the library reserves statically on every device where it is
 * loaded, until the process exits.  The first call on each device resolves
 * that array's address (cudaGetSymbolAddress) and must precede any stream
 * capture.  All calls share the array: calls that overlap on the GPU race.
 * A plan whose single image needs more than 16 MiB of scratch is rejected
 * with FFB_ERR_UNSUPPORTED (not reached for L <= 512).  Arguments as
 * ffb_polar; the plan must already exist. */
int ffb_polar_noalloc(ffb_plan_t plan, const float *d_images, int64_t n, float *d_F,
                      void *stream);

/* ffb_expand -- Alg. 1 steps 3-4: a = T* I for n images.
 * d_images [n][L][L] float32 -> d_coef [n][P][2] float32 (layout above).
 * Eq. nufft by NUFFT, Eq. 1DFFT by FFT on each ring, Eq. a as a grouped
 * contraction over k in the plan's precision.  n >= 0 (n = 0 is a no-op). */
int ffb_expand(ffb_plan_t plan, const float *d_images, int64_t n, float *d_coef,
               void *stream);

/* ffb_expand_adjoint -- the exact adjoint T y = Re(M^H y) of ffb_expand for
 * the inner products Re sum conj(u) v (coefficients) and sum x y (images):
 * transposed radial quadrature, conjugate ring DFT, type-1 NUFFT, real part.
 * d_coef [n][P][2] -> d_images [n][L][L].  The synthesis of a real image from
 * its coefficients is ffb_expand_adjoint applied to W a with W = 1 (k = 0),
 * 2 (k > 0). */
int ffb_expand_adjoint(ffb_plan_t plan, const float *d_coef, int64_t n,
                       float *d_images, void *stream);

/* ffb_covariance -- Alg. 2 steps 1-4 (accumulation part): adds n coefficient
 * vectors to the plan's float64 accumulator of the k = 0 mean (Eq. mean2) and
 * of the blocks sum_i Re{a_k a_k^*} (Eqs. ck, ck_0).  reset != 0 clears it
 * first.  Streaming over several calls gives the same result as one call. */
int ffb_covariance(ffb_plan_t plan, const float *d_coef, int64_t n, int reset,
                   void *stream);

/* ffb_cov_get -- finalises the accumulator: d_mean0[p_0] = (1/n) sum a_{0,q},
 * d_C = packed blocks C^(k) (k ascending, each p_k x p_k row-major float64),
 * C^(k) = (1/n) Re{A A^*} with the k = 0 block centred (Eqs. ck, ck_0).
 * Either pointer may be NULL.  Synchronises the stream; returns latched
 * device errors. */
int ffb_cov_get(ffb_plan_t plan, double *d_mean0, double *d_C, void *stream);

/* Covariance statistics of disjoint image sets (e.g. one per GPU; Sec. IV
 * splits the images over workers).  A state is the float64 host vector
 * [n, mean0 (p_0 values), C^(0..k_max) packed as in ffb_cov_get]
 * (length 1 + p_0 + sum p_k^2).
 * ffb_cov_export: finalises the plan's accumulator into h_state (synchronises).
 * ffb_cov_merge:  host-only; pools nstates consecutive states of the plan
 *   sizes (k_max, h_p[k_max+1]) into h_out: n = sum n_r, m = sum n_r m_r / n,
 *   C^(0) = sum n_r (C0_r + (m_r - m)(m_r - m)^T)/n, C^(k) = sum n_r C^(k)_r/n.
 * ffb_cov_import: replaces the plan's accumulator by a (pooled) state, so that
 *   ffb_cov_get / ffb_eig return the pooled covariance (synchronises). */
int ffb_cov_export(ffb_plan_t plan, double *h_state, void *stream);
int ffb_cov_merge(int k_max, const int *h_p, int nstates, const double *h_states, double *h_out);
int ffb_cov_import(ffb_plan_t plan, const double *h_state, void *stream);

/* ffb_ringdft_table -- host only: the tables of the ring DFT that runs on the
 * tensor cores (Eq. 1DFFT at n_theta = 512 with BF16x3), as float copies of
 * their bf16 hi and lo parts: [parity p][192 columns][n_theta/2], column
 * 2e + c (c = 0 real, 1 imaginary part) of k = 2e + p, zero for k > k_max.
 * With the ring's conjugate completion and samples f_l = u_l + i v_l
 * (l < n_theta/2), F_k = sum_l T[p=0][2e+c][l] u_l (even k) or
 * sum_l T[p=1][2e+c][l] v_l (odd k), T = hi + lo, which includes the
 * 2 pi / n_theta weight and the factor 2 of the completion.  h_hi, h_lo:
 * 2 x 192 x n_theta/2 floats each (either may be NULL).  Returns
 * FFB_ERR_UNSUPPORTED for odd n_theta or k_max >= 192. */
int ffb_ringdft_table(int n_theta, int k_max, float *h_hi, float *h_lo);

/* ffb_expand_cov_host -- Alg. 1 steps 3-4 and the accumulation of Alg. 2
 * steps 1-4 for n images held in HOST memory, with the statistics returned
 * to host memory: the end-to-end call of a user whose image stack sits in
 * host RAM.  h_images [n][L][L] float32 (page-locked memory gives the full
 * copy bandwidth; pageable memory works at the driver's staged rate).  The
 * images move to the device in parts of whole chunks through a ring of
 * three device buffers on a copy stream of the plan, each copy overlapping
 * the expansion of the part before it; every part is expanded as ffb_expand
 * and added to the accumulator as ffb_covariance (reset != 0 clears it
 * first, so reset = 0 continues an earlier accumulation).  Then, when h_mean0
 * or h_C is not NULL, the accumulator is finalised as ffb_cov_get and the
 * k = 0 mean (p_0 float64) and the packed blocks (sum p_k^2 float64) are
 * copied to them.  The device buffers (three parts of at most 256 MiB of
 * images, and the coefficients of one part: P / (2 L^2) times as many bytes
 * as its images) are allocated on first use and kept by the plan.  Synchronises `stream`; returns latched
 * device errors, FFB_ERR_STATE when statistics are asked for and nothing was
 * accumulated.  The host buffer must stay valid until the call returns. */
int ffb_expand_cov_host(ffb_plan_t plan, const float *h_images, int64_t n, int reset,
                        double *h_mean0, double *h_C, void *stream);

/* ffb_eig -- Alg. 2 step 4: eigenpairs of every block C^(k) by a batched
 * float64 cyclic Jacobi solver on the GPU (one CTA per block).
 * d_evals[P]: per block descending; d_evecs packed p_k x p_k row-major,
 * column l = u^(k)_l, each signed so its largest-magnitude entry (first on
 * ties) is positive.  Either pointer may be NULL.  Synchronises the stream. */
int ffb_eig(ffb_plan_t plan, double *d_evals, double *d_evecs, void *stream);

/* ffb_eig_blocks -- the same batched float64 Jacobi solver applied to caller
 * supplied symmetric blocks: d_C packed like ffb_cov_get's output (k
 * ascending, p_k x p_k row-major).  Outputs as ffb_eig.  Synchronises. */
int ffb_eig_blocks(ffb_plan_t plan, const double *d_C, double *d_evals, double *d_evecs,
                   void *stream);

/* ffb_radial_eigenfunctions -- Alg. 2 step 5 (Eq. sPCArad) in float64 from
 * the eigenvectors of the last ffb_eig / ffb_eig_blocks / ffb_denoise:
 * f^{k,l}(xi_j) = sum_q N_{k,q} J_k(R_{k,q} xi_j / c) u^(k)_l(q), written to
 * d_f[offset[k] * n_xi + j * p_k + l] (n_xi * P values).  Asynchronous. */
int ffb_radial_eigenfunctions(ffb_plan_t plan, double *d_f, void *stream);

/* ffb_eigenimages -- the steerable principal components on the pixel grid
 * (Sec. V, built from Eq. IFT_FB): g^{k,l}(r, phi) = sum_q u^(k)_l(q)
 * F^{-1}(psi^{k,q})(r, phi), complex, for npairs pairs (h_k[i], h_l[i]) (host
 * arrays), written as d_out[i][a1][a2][re, im] float64.  The phase factor is
 * i^k (as derived from Eq. IPFT; the printed equation has i^{-k}).  For k > 0
 * the real and imaginary parts are the two real eigenimages of the pair.
 * Synchronises. */
int ffb_eigenimages(ffb_plan_t plan, int npairs, const int *h_k, const int *h_l, double *d_out,
                    void *stream);

/* ffb_select -- Sec. V component selection from the eigenpairs of the last
 * ffb_eig/ffb_denoise call: gains h^(k)_l per ffb_denoise_mode (K pairs for
 * TOPK, noise variance sigma2 and image count n for MP_WIENER), stored in the
 * plan together with the filter matrices M^(k) = U^(k) diag(h^(k)) U^(k)T
 * used by ffb_filter.  Optionally copies the gains to h_gain[P] (host, may be
 * NULL).  Synchronises. */
int ffb_select(ffb_plan_t plan, int mode, int K, double sigma2, int64_t n, double *h_gain,
               void *stream);

/* ffb_filter -- applies the selected steerable filter to coefficients:
 * a_out^(k) = M^(k) (a^(k) - m) + m with m the k = 0 mean (Alg. 2 step 1),
 * i.e. the projection / shrinkage of c_{k,l} = sum_q a_{k,q} u_l(q)
 * (Eq. sPCAcoeff) mapped back to the Fourier-Bessel basis.
 * flags bit 0 (FFB_FILTER_LINEAR): drop the mean terms (the linear part,
 * which is also the map's own transpose); bit 1 (FFB_FILTER_WEIGHT): multiply
 * the result by W (1 for k = 0, 2 for k > 0).  In place allowed.  Requires a
 * prior ffb_select. */
int ffb_filter(ffb_plan_t plan, const float *d_coef_in, int64_t n, float *d_coef_out, int flags,
               void *stream);
#define FFB_FILTER_LINEAR 1
#define FFB_FILTER_WEIGHT 2

/* ffb_weight -- d_out = W a (W = 1 on k = 0 coefficients, 2 on k > 0), the
 * weights that turn the adjoint into the synthesis of a real image from its
 * k >= 0 coefficients.  In place allowed. */
int ffb_weight(ffb_plan_t plan, const float *d_coef_in, int64_t n, float *d_coef_out, void *stream);

/* ffb_denoise -- expansion, steerable covariance, eigendecomposition,
 * selection (ffb_denoise_mode; K pairs for TOPK, sigma2 the noise variance
 * for MP_WIENER), filtering of c_{k,l} = sum_q a_{k,q} u_l(q) (Eq. sPCAcoeff)
 * and synthesis back to images through the adjoint with weights W.
 * d_images [n][L][L] -> d_out [n][L][L].  Uses and overwrites the plan's
 * covariance accumulator.  Synchronises the stream. */
int ffb_denoise(ffb_plan_t plan, const float *d_images, int64_t n, int mode,
                int K, double sigma2, float *d_out, void *stream);

/* ffb_sync -- waits for the stream and returns the first latched device error
 * (then clears it). */
int ffb_sync(ffb_plan_t plan, void *stream);

/* ffb_profile -- per-launch timing: enable = 0 turns it off; enable = s >= 1
 * brackets every s-th launch of each kernel class (the first included) by two
 * CUDA events on its stream (s = 1: every launch; a larger stride keeps the
 * events' own cost out of a timed run).  Enabling discards earlier records.
 * FFB_ERR_ARG for enable < 0. */
int ffb_profile(ffb_plan_t plan, int enable);

/* ffb_profile_read -- per kernel class: h_ms[16] the launches' total duration
 * in milliseconds (with a stride s > 1 the mean of the timed launches times
 * the launch count), h_calls[16] the launches since profiling was enabled;
 * then discards the records.  Classes: 0 rows FFT, 1 column FFT, 2 interpolation + ring DFT,
 * 3 radial quadrature, 4 covariance, 5 covariance shift/finalise, 6 Jacobi,
 * 7 transposed quadrature, 8 inverse ring DFT + spreading, 9 inverse column
 * FFT, 10 inverse row FFT + deconvolution, 11 steerable filter, 12 setup,
 * 13 shared-memory grid + interpolation, 14 ring FFT from the polar buffer,
 * 15 adjoint spreading in shared memory.
 * Synchronises on the recorded events. */
int ffb_profile_read(ffb_plan_t plan, double *h_ms, int64_t *h_calls);

/* ffb_invariants -- rotation-invariant features of n images from their
 * steerable PCA coefficients c_{k,l} = u^(k)_l^T (a^(k) - mean [k = 0])
 * (Eq. sPCAcoeff, eigenpairs and k = 0 mean of the last ffb_eig / ffb_svd):
 * the bispectrum-like features of Sec. I.
 *   power:      d_pow[i][t] = |c_{k,l}|^2 for the npow pairs h_pairs[t] = (k, l);
 *   bispectrum: d_bis[i][t] = c_{k1,l1} c_{k2,l2} conj(c_{k1+k2,l3}) (complex,
 *               [re, im]) for the nbis quintuples h_triples[t] = (k1, l1, k2, l2, l3).
 * An in-plane rotation multiplies c_{k,l} by e^{-ik alpha}, which cancels in
 * both; a reflection leaves the power and conjugates the bispectrum.
 * d_coef: device [n][P][2]; d_pow float32 [n][npow]; d_bis float32
 * [n][nbis][2]; index lists are host arrays (FFB_ERR_ARG for a pair outside
 * the basis or k1 + k2 > k_max; FFB_ERR_STATE before any eigendecomposition).
 * Synchronises. */
int ffb_invariants(ffb_plan_t plan, const float *d_coef, int64_t n, int npow, const int *h_pairs, float *d_pow,
                   int nbis, const int *h_triples, float *d_bis, void *stream);

/* ffb_svd -- Alg. 2 step 4 by the SVD route of Sec. III: the eigenpairs of every
 * C^(k) from the coefficient matrices of n images (d_coef: device [n][P][2])
 * without forming the covariance from the data.  For each k, X_k stacks the
 * rows (Re a_{i,k,.}, Im a_{i,k,.}) (k > 0) or Re a_{i,0,.} - mean (k = 0);
 * a tall-skinny QR X_k = Q_k R_k (float32 Householder in shared memory,
 * float64 norms, per image range and then merged) is followed by the float64
 * Jacobi eigensolver on R_k^T R_k / n, whose eigenvectors are the singular
 * vectors of A^(k) and eigenvalues s^2 / n.  Outputs as ffb_eig (device,
 * may be NULL); the plan's eigenpairs, k = 0 mean and finalised covariance
 * (R^T R / n) are replaced, so ffb_select / ffb_filter / ffb_radial_* use
 * them.  Requires p_k <= 128 (FFB_ERR_UNSUPPORTED otherwise); synchronises. */
int ffb_svd(ffb_plan_t plan, const float *d_coef, int64_t n, double *d_evals, double *d_evecs, void *stream);

/* ffb_estimate_support -- radius of compact support R and band limit c of a
 * stack, estimated from the noisy images (the procedure of Sec. V applied to
 * the simulated ribosome projections).  Real domain: subtract the mean image,
 * average the per-pixel variance over rings r = round(|i|) < L/2 (the mean
 * radial variance), subtract the noise variance, clip at zero and accumulate
 * with the weight r; R is the first ring at which the cumulative sum reaches
 * `frac` (0 < frac <= 1, the paper uses 0.999) of its total.  Fourier domain:
 * the same with the angular average of the mean power spectrum
 * (1/L^2) |F(I - mean)(xi_j, theta_l)|^2 on the plan's polar grid and the
 * weight xi_j w_j; c is the node xi_j reached.  Use a plan with c = 1/2 and
 * R = L/2 so that the polar grid spans the whole band.  sigma2 >= 0 is the
 * noise variance; sigma2 < 0 estimates it as the mean variance of the pixels
 * with |i| >= L/2.  Outputs (host): h_out[4] = {R in pixels, c in cycles per
 * pixel, the noise variance used, index of c's node}; h_radvar[L/2] the mean
 * radial variance, h_radpow[n_xi] the radial power spectrum (both may be
 * NULL).  d_images: device [n][L][L], n >= 1.  Allocates and frees its own
 * scratch on `stream` and synchronises it. */
int ffb_estimate_support(ffb_plan_t plan, const float *d_images, int64_t n, double frac, double sigma2,
                         double *h_out, double *h_radvar, double *h_radpow, void *stream);

/* Number of kernel launches issued by this plan since creation (for
 * accounting of GPU work).  Launches replayed from a group's CUDA graph are
 * counted on the plan whose stack they belong to. */
int64_t ffb_launch_count(ffb_plan_t plan);

/* ---- batching: many stacks of uneven L and n ----------------------------
 * Sec. IV notes that the expansion and the covariance are sums over images
 * that may be split among workers.  A group runs S independent stacks
 * (1 <= S <= 64), each with its own plan, through a1-a7 in one call:
 *   - each stack's expansion (a1-a4) runs on its own branch stream; with a
 *     tensor-core precision the call proceeds in rounds, round r taking the
 *     r-th group of chunks of every stack that has one (the chunks one
 *     quadrature launch of ffb_expand would take), and the radial quadrature
 *     (a5, Eq. a) of a round is ONE persistent launch over the (stack, k,
 *     M tile) items of all its stacks: a grouped GEMM over the uneven
 *     p_k x n_xi blocks of every stack, the stacks' TMA descriptors in
 *     device memory (FFB_FP32 plans run a5 per stack on their branches);
 *   - the covariance of all stacks (a6/a7) is ONE persistent launch over the
 *     (stack, k block, image range) items of every stack: a grouped SYRK over
 *     the uneven per-k block sizes p_k (tensor cores in the plans' precision,
 *     or float32 tiles for FFB_FP32), plus one launch of the k = 0 sums;
 *   - the first call with a given set of pointers, sizes and reset flags runs
 *     eagerly; once per group it also times the candidate item shapes of the
 *     grouped launch (images per item, images per tensor-core tile, grid) on
 *     that call's coefficients, accumulating into scratch, and keeps the
 *     fastest (ffb_group_tuning lists them), and times the launch shapes of
 *     the grouped quadrature (CTAs per SM, pipeline stages) on the call's
 *     first round (ffb_group_quad_tuning); the second call with the same
 *     arguments captures the launches into a CUDA graph; later ones replay it.
 * Results are those of ffb_expand + ffb_covariance on each plan: the same
 * coefficients bit for bit; the covariance accumulated in another order.
 * The plans stay owned by the caller and must outlive the group; they must
 * be distinct, share one precision (ffb_set_precision on a member afterwards
 * makes the group's calls return FFB_ERR_STATE), and with a tensor-core
 * precision every p_k must be <= 128 (FFB_ERR_UNSUPPORTED otherwise).  While
 * a group call is in flight its plans must not be used on other streams. */
typedef struct ffb_group_s *ffb_group_t;

/* ffb_group_create -- allocates each plan's scratch, the branch streams and
 * the tuner's scratch accumulator; synchronises `stream`. */
int ffb_group_create(ffb_group_t *out, int S, const ffb_plan_t *plans, void *stream);
int ffb_group_destroy(ffb_group_t group);

/* ffb_group_expand_cov -- for every stack s with h_n[s] > 0: expand the
 * images h_images[s] (device [h_n[s]][L_s][L_s]) into h_coef[s] (device
 * [h_n[s]][P_s][2]) and add them to the stack's covariance (restarted first
 * when reset != 0).  h_images, h_n, h_coef are host arrays of S entries; a
 * stack with h_n[s] == 0 is skipped (its pointers may be NULL).  Asynchronous
 * on `stream`; device errors are returned by ffb_group_sync or by the plans'
 * synchronising calls (ffb_cov_get, ffb_eig). */
int ffb_group_expand_cov(ffb_group_t group, const float *const *h_images, const int64_t *h_n,
                         float *const *h_coef, int reset, void *stream);

/* ffb_group_covariance -- a6/a7 only, for coefficients already computed
 * (h_coef[s]: device [h_n[s]][P_s][2]), as one grouped launch. */
int ffb_group_covariance(ffb_group_t group, const float *const *h_coef, const int64_t *h_n, int reset,
                         void *stream);

/* ffb_group_sync -- synchronises `stream` and returns the first device error
 * of the grouped launches or of any member plan. */
int ffb_group_sync(ffb_group_t group, void *stream);

/* ffb_group_info -- h_info[14]: S, precision, tuned images per item, tuned
 * images per tensor-core tile, tuned grid (CTAs), graphs instantiated, graph
 * replays, eager calls, kernel launches of the last call, tuning candidates;
 * then for the grouped quadrature: tuned CTAs per SM, tuned pipeline stages,
 * its tuning candidates, grouped quadrature launches (rounds) of the last
 * call shape (0 for FFB_FP32 groups). */
int ffb_group_info(ffb_group_t group, int64_t *h_info);

/* ffb_group_quad_tuning -- the timed launch shapes of the grouped quadrature
 * (up to max): CTAs per SM, pipeline stages, milliseconds of one launch on
 * the first round of the tuning call.  Returns the number written (a
 * negative ffb_status on error). */
int ffb_group_quad_tuning(ffb_group_t group, int max, int *h_per_sm, int *h_stages, float *h_ms);

/* ffb_group_tuning -- the timed candidates (up to max): images per item,
 * images per tile, grid, milliseconds of one grouped launch.  Returns the
 * number written (a negative ffb_status on error). */
int ffb_group_tuning(ffb_group_t group, int max, int *h_per, int *h_tile, int *h_grid, float *h_ms);

const char *ffb_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* FFB_H */
