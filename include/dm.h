/*
 * dm.h -- C ABI of the GB300 DeepMatching hot path.
 *
 * DeepMatching (Revaud, Weinzaepfel, Harchaoui, Schmid) matches two images
 * I (W1 x H1) and I' (W2 x H2) -- Sec. 3.1 -- and returns quasi-dense
 * correspondences (p, p', s): p the centre of a 4x4 atomic patch of I, p' a
 * pixel of I', s a score -- Eq. 16.  The calls below are the steps of that
 * computation:
 *
 *   dm_descriptors        per-pixel 9-D descriptors (Sec. 3.2 "Pixel descriptor")
 *   dm_correlate_pyramid  bottom-level correlation (Eq. 3-4) and the
 *                         multi-level correlation pyramid (Eq. 5-12, Algorithm 1)
 *   dm_backtrack          backtracking with merging (Eq. 13-15) and reciprocal
 *                         verification (Eq. 16)
 *   dm_match              all of the above
 *
 * and the paper's extensions built on them:
 *
 *   dm_prototypes, dm_correlate_pyramid_approx   approximate form (Sec. 4.1)
 *   dm_match_invariant    scale and rotation invariant form (Sec. 4.2, Algorithm 2)
 *   dm_match_star, dm_backtrack_star             DM*, the earlier backtracking (Sec. 5.3)
 *   dm_deepflow           DeepFlow, the variational flow fed by the matches (Sec. 4.3)
 *   dm_loss_grad          differentiable form (a loss the paper does not define)
 *   dm_match_batch        many pairs in concurrent lanes (CUDA-graph capturable)
 *
 * Conventions shared by every call:
 *   - Pointers named d_* are CUDA device pointers on the context's device;
 *     h_* are host pointers.  The caller owns every buffer and the stream; the
 *     library never allocates device memory.  Workspace sizes come from
 *     dm_workspace_bytes(); a workspace must be 256-byte aligned.
 *   - Images are float32, row-major [H][W], values in [0, 1].  Descriptors
 *     are float32 [H][W][9] (8 orientation channels, then the mu channel).
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) unless stated otherwise; argument errors are reported
 *     synchronously and nothing is launched.  A failure of a CUDA call returns
 *     DM_ECUDA.  dm_last_error() describes the last failure of a context.
 *   - Devices: each call makes the context's device current for its duration
 *     and restores the caller's current device.
 */
#ifndef DM_H
#define DM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DM_OK = 0,
    DM_EINVAL = 1,        /* bad argument (size, pointer, alignment, capacity)     */
    DM_ENOMEM = 2,        /* workspace smaller than dm_workspace_bytes() requires  */
    DM_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed           */
    DM_ETIMEOUT = 4,      /* a bounded device-side wait gave up                    */
    DM_EUNSUPPORTED = 5,  /* valid request this build does not handle              */
    DM_EOVERFLOW = 6      /* output or frontier capacity exceeded                  */
} dm_status;

typedef enum {
    DM_FP32 = 0,          /* FP32 everywhere; bit-exact with the FP32 reference    */
    DM_BF16 = 1,          /* bottom-level correlation on BF16 tensor cores (FP32
                             accumulation); the rest of the pyramid in FP32         */
    DM_FP8_E4M3 = 2       /* bottom-level correlation on FP8 (E4M3) tensor cores:
                             each patch vector of I scaled by its own power of two
                             so that its largest entry lies in [224, 448], the
                             descriptors of I' scaled by 256; FP32 accumulation,
                             scales undone before the power; the rest in FP32     */
} dm_precision;

/* Parameters of the method.  Defaults (dm_config_default) are the paper's:
 * nu1 = nu2 = nu3 = 1, slope (varsigma) = 0.2, mu = 0.3 (Sec. 5.2 "Pixel
 * descriptor parameters"), lambda = 1.4 (Sec. 5.2 "Non-linear rectification"),
 * image_scale = 255 (input in [0,1] is mapped to 0..255 before the gradient). */
typedef struct {
    float nu1, nu2, nu3;   /* std. dev. of the three Gaussian smoothings (0 = none) */
    float slope;           /* sigmoid slope varsigma                               */
    float mu;              /* ninth, constant descriptor component                 */
    float lambda;          /* rectification exponent (Eq. 11)                      */
    float image_scale;     /* multiplier applied to input intensities              */
    int precision;         /* dm_precision                                         */
    int compensated;       /* 1 (default): the 4-child sums of the pyramid (Eq. 12)
                              are Knuth-TwoSum compensated, rounded once; 0: plain
                              FP32 sums in child order.  Path scores (Eq. 14) are
                              always exact: terms rounded to multiples of 2^-28,
                              summed in 32-bit fixed point, rounded to FP32 once */
} dm_config;

/* One output correspondence (Eq. 16): (x1, y1) is the centre of an atomic
 * patch of I, (x2, y2) the matched pixel of I', score the sum of the
 * correlations along its backtracking path (Eq. 14). */
typedef struct {
    float x1, y1, x2, y2, score;
} dm_match_t;

typedef struct dm_ctx dm_ctx;          /* host-side state: config, device, last error */
typedef struct dm_pyramid dm_pyramid;  /* host-side view of a pyramid in a workspace  */

/* Status word values written by the device into the workspace (dm_read_status). */
#define DM_DEV_OK 0
#define DM_DEV_FRONTIER_OVERFLOW 1     /* a merge table filled up during backtracking */
#define DM_DEV_OUTPUT_OVERFLOW 2       /* more matches than the output capacity       */
#define DM_DEV_TIMEOUT 4               /* a bounded wait inside a pyramid kernel gave up */

/* Fill *cfg with the paper's parameters, DM_FP32 and compensated = 1. */
void dm_config_default(dm_config* cfg);

/* Create a context bound to CUDA device `device`.  Host allocation only. */
dm_status dm_create(const dm_config* cfg, int device, dm_ctx** out);
dm_status dm_destroy(dm_ctx* ctx);
/* Text of the last failure on ctx ("" if none); owned by ctx. */
const char* dm_last_error(const dm_ctx* ctx);

/* Geometry of the method for a pair of sizes (Sec. 3.2 and Algorithm 1):
 *   *L        top level: min{l : 4*2^l >= max(W1,H1)} (where Algorithm 1 stops),
 *             lowered to the highest level at which image 1 has a patch (a wide,
 *             low image has none at that level: e.g. 1242 x 375 gives 8, not 9)
 *   *n_patch0 atomic patches (centres 4k+2 inside I)
 *   *n_patch  lattice patches of levels >= 1 (centres in 4Z^2 inside I)
 *   dw, dh    (may be NULL) map domain of level l = 0..L+1: ceil(W2/2^l) x ceil(H2/2^l)
 * Requires W1, H1 >= 4, max(W1, H1) >= 5, W2, H2 >= 1; DM_EUNSUPPORTED when
 * L > 14 (the fixed-point path scores hold L + 1 terms in 32 bits) or the
 * atomic indices (pixel of I', patch * 16 + offset) exceed 32 bits.  Sizes
 * whose merge keys patch * |domain| + position exceed 32 bits are supported
 * with 64-bit keys (dm_set_merge_keys). */
dm_status dm_geometry(int W1, int H1, int W2, int H2, int* L, int* n_patch0, int* n_patch, int* dw, int* dh);

/* Workspace bytes for a pair of sizes:
 *   desc_bytes      scratch of dm_descriptors for the larger image
 *   pyramid_bytes   dm_correlate_pyramid
 *   backtrack_bytes dm_backtrack
 *   match_bytes     dm_match (descriptors of both images + the above)
 * Any pointer may be NULL. */
dm_status dm_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* desc_bytes,
                             size_t* pyramid_bytes, size_t* backtrack_bytes, size_t* match_bytes);

/* Pixel descriptors of one image (Sec. 3.2 "Pixel descriptor"):
 * Gaussian smoothing (nu1) of image_scale * I, central-difference gradient,
 * non-negative projections on the 8 directions k*pi/4, smoothing (nu2),
 * sigmoid x -> 2/(1+exp(-slope x)) - 1, smoothing (nu3), then the 8 channels
 * and mu are L2-normalised together.  Smoothings: std. dev. nu, taps on
 * [-ceil(3 nu), ceil(3 nu)] normalised to 1, replicated border.
 * d_img [H][W] float32; d_desc [H][W][9] float32 (output); d_tmp scratch of
 * at least desc_bytes (dm_workspace_bytes with this W, H as image 1). */
dm_status dm_descriptors(dm_ctx* ctx, const float* d_img, int W, int H, float* d_desc, void* d_tmp,
                         size_t tmp_bytes, void* stream);

/* Bottom-up correlation pyramid (Algorithm 1).
 * Level 0 (Eq. 3-4): C0(p, t) = (1/16) sum over the 4x4 window of the 9-D
 * dot products between the atomic patch of I centred at p and the window
 * [t-2, t+1]^2 of I' (zero descriptors outside the images).  Each level l is
 * stored max-pooled and subsampled (Eq. 8-9) after rectification (Eq. 11):
 * P_l(p, r) = (max over the in-domain points 2r+m, m in {-1,0,1}^2, of C_l)^lambda
 * with the argmax code (my+1)*3 + (mx+1).  Level l >= 1 (Eq. 12): C_l(p, q) =
 * mean over the existing children i of P_{l-1}(p + 2^l o_i, q + o_i) (0 outside
 * the domain); the top level C_L is stored unpooled.
 * The pyramid lives in d_ws (>= pyramid_bytes); *out is a host handle that
 * references it (free with dm_pyramid_free; it does not own d_ws). */
dm_status dm_correlate_pyramid(dm_ctx* ctx, const float* d_desc1, int W1, int H1, const float* d_desc2, int W2,
                               int H2, void* d_ws, size_t ws_bytes, dm_pyramid** out, void* stream);

/* Approximate DeepMatching (Sec. 4.1): image 1's atomic patches replaced by
 * their closest prototype from a dictionary of D learned per pair.
 *
 * dm_prototypes: the dictionary, by k-means of the atomic patches of image 1
 * (their 144-vectors a[(dy*4 + dx)*9 + c] over the Eq. 3-4 window, zero
 * outside I) with every centroid projected back on the hypersphere of the
 * patches (norm 4) after each update.  Start: centroid d = patch h_init[d]
 * projected (h_init: D host ints in [0, P0); NULL = patches floor(d P0 / D)).
 * One iteration: assign every patch to the closest centroid (largest dot
 * product, ties to the lower index), then replace each centroid by the sum of
 * its members projected to norm 4 (a centroid without members is kept).
 * After `iters` iterations (>= 0) a last assignment is made.  Out: d_protos
 * [D][144] (FP32) and d_assign [P0] (prototype of each atomic patch, int32).
 * The member sums are exact fixed-point sums, so the result does not depend
 * on the order of the atomic updates.  D in [1, P0] (P0 = dm_geometry's
 * n_patch0); d_ws >= dm_prototypes_workspace_bytes.  h_init is copied from
 * pageable memory on `stream` (not capturable in a CUDA graph).
 *
 * dm_correlate_pyramid_approx: the pyramid of dm_correlate_pyramid with atomic
 * patch p of image 1 replaced by d_protos[d_assign[p]]: level 0 is computed
 * and stored once per prototype (D maps instead of P0), and the level-1 and
 * backtracking steps read the map of each atomic child through d_assign.
 * W1, H1 give image 1's size (its descriptors are not needed).  d_protos and
 * d_assign stay caller-owned and must stay unchanged while the pyramid is used
 * (dm_backtrack reads d_assign); entries of d_assign outside [0, D) are
 * clamped to that range.  Same workspace as dm_correlate_pyramid;
 * dm_pyramid_level reports n_patches = D for level 0.  Results equal those of
 * dm_correlate_pyramid on descriptors whose atomic patches are the assigned
 * prototypes.  dm_loss_grad refuses such a pyramid (DM_EUNSUPPORTED). */
dm_status dm_prototypes_workspace_bytes(dm_ctx* ctx, int W1, int H1, int D, size_t* bytes);
dm_status dm_prototypes(dm_ctx* ctx, const float* d_desc1, int W1, int H1, int D, int iters, const int* h_init,
                        float* d_protos, int* d_assign, void* d_ws, size_t ws_bytes, void* stream);
dm_status dm_correlate_pyramid_approx(dm_ctx* ctx, const float* d_protos, int D, const int* d_assign, int W1, int H1,
                                      const float* d_desc2, int W2, int H2, void* d_ws, size_t ws_bytes,
                                      dm_pyramid** out, void* stream);

/* Device views of one level of a pyramid (valid after the producing stream
 * work completes).  level in [0, L]; for level < L: d_vals = P_l
 * [n_patches][mh][pitch] (columns mw..pitch-1 are row padding, not data) and
 * d_argmax its codes in the same layout; for level == L: d_vals = C_L
 * [n_patches][mh][mw] (pitch = mw) and d_argmax = NULL.  d_valid [n_patches]:
 * 1 if the patch exists (Eq. 7 with the boundary rule).  Pooled rows are
 * padded to a multiple of 16 values so that every row starts 16-byte aligned.
 * Any output pointer may be NULL. */
dm_status dm_pyramid_level(const dm_pyramid* pyr, int level, const float** d_vals, const unsigned char** d_argmax,
                           const unsigned char** d_valid, int* n_patches, int* mw, int* mh, int* pitch);
dm_status dm_pyramid_free(dm_pyramid* pyr);

/* Backtracking (Eq. 13-15) from every top-level position (Sec. 3.3 "Merging
 * correspondences"), merging tuples equal in (level, patch, position) by
 * their highest score, then reciprocal verification (Eq. 16): the best tuple
 * of each atomic patch is kept iff it is also the best tuple whose pixel
 * lies in its 4x4 cell of I' (ties: higher score, then lower index).
 * d_out receives up to `capacity` matches in atomic-patch order; *d_count
 * (device int) the number found (may exceed capacity: then
 * DM_DEV_OUTPUT_OVERFLOW is set in the status word).  d_ws >= backtrack_bytes. */
dm_status dm_backtrack(dm_ctx* ctx, const dm_pyramid* pyr, void* d_ws, size_t ws_bytes, dm_match_t* d_out,
                       int capacity, int* d_count, void* stream);

/* Whole method on device buffers: descriptors of both images, pyramid,
 * backtracking.  d_ws >= match_bytes. */
dm_status dm_match(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                   void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count, void* stream);

/* Whole method on host buffers: copies h_img1/h_img2 to the device (into
 * d_ws), runs dm_match, copies the matches and their count back, and
 * synchronises `stream`.  h_out holds `capacity` entries; *h_count receives
 * the number of matches found.  Pinned host memory gives asynchronous copies. */
dm_status dm_match_host(dm_ctx* ctx, const float* h_img1, int W1, int H1, const float* h_img2, int W2, int H2,
                        void* d_ws, size_t ws_bytes, dm_match_t* h_out, int capacity, int* h_count, void* stream);

/* DeepFlow (Sec. 4.3): dense flow (u, v) from I1 to I2 (same size W x H,
 * values in [0,1]) refining the matches with a variational energy: data term
 * delta Psi(theta0 (grad3 I . w)^2) + gamma Psi(normalised gradient
 * constancy), smoothness alpha(x) Psi(|grad u|^2 + |grad v|^2) with alpha =
 * exp(-kappa |grad I1|), matching term beta_k c phi Psi(|w - w'|^2) with phi
 * from the structure tensor and the appearance difference at each match,
 * Psi(s^2) = sqrt(s^2 + eps^2); coarse to fine (factor eta, levels down to a
 * side of min_size) with warping, n_fixed fixed-point steps per level of
 * n_sor red-black SOR sweeps each (relaxation omega).  Defaults
 * (dm_flow_params_default) are the paper's: sigma 0.5, eta 0.95, gamma 0.8,
 * delta 0, beta 300, b 0.6, kappa 5, zeta 0.1, eps 0.001, sigma_M 50, 5 x 25
 * iterations; omega 1.6 and min_size 16 are this library's choices.
 * d_matches: device array of `capacity` matches, of which *d_count (device
 * int) are used -- the output of dm_match can be passed as it is, so the two
 * calls chain on one stream without a host round trip; d_matches / d_count
 * may be NULL (no matching term).  d_u, d_v: device [H][W] outputs.
 * d_ws >= dm_deepflow_workspace_bytes (256-byte aligned).  No host
 * synchronisation; the call can be captured in a CUDA graph. */
typedef struct {
    double sigma, eta, gamma, delta, beta, b, kappa, zeta, eps, sigma_m, omega, image_scale;
    int n_fixed, n_sor, min_size;
} dm_flow_params;
void dm_flow_params_default(dm_flow_params* p);
dm_status dm_deepflow_workspace_bytes(dm_ctx* ctx, int W, int H, int capacity, const dm_flow_params* prm,
                                      size_t* bytes);
dm_status dm_deepflow(dm_ctx* ctx, const float* d_img1, const float* d_img2, int W, int H, const dm_match_t* d_matches,
                      const int* d_count, int capacity, const dm_flow_params* prm, float* d_u, float* d_v, void* d_ws,
                      size_t ws_bytes, void* stream);

/* DM*, the earlier backtracking variant compared in Sec. 5.3 (Table
 * "oldvsnew"): entry points are the local maxima of the maps C_l(p, .) of every
 * level l = 1..L (q is one iff C_l(p, q) > 0, C_l(p, q) > C_l(p, r) for its
 * in-domain 8-neighbours r before q in row-major order and >= for those
 * after it), each with start score C_l(p, q); a tuple carries its start score
 * down unchanged (Eq. 13 children, merged by the highest start), and an
 * atomic correspondence scores start + the rectified atomic correlation at
 * its end (P_0 at the last step).  Reciprocal verification and output as
 * dm_backtrack / dm_match.  dm_backtrack_star takes a pyramid built by a
 * context with the same parameters as ctx (lambda is the context's);
 * d_ws >= backtrack_bytes of dm_star_workspace_bytes.  dm_match_star runs the
 * whole chain; d_ws >= match_bytes.  The tables of DM* also hold the entry
 * points, so its workspaces are larger than dm_backtrack's / dm_match's.
 * dm_read_status works on both workspaces. */
dm_status dm_star_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* backtrack_bytes,
                                  size_t* match_bytes);
dm_status dm_backtrack_star(dm_ctx* ctx, const dm_pyramid* pyr, void* d_ws, size_t ws_bytes, dm_match_t* d_out,
                            int capacity, int* d_count, void* stream);
dm_status dm_match_star(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                        void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count, void* stream);

/* Scale and rotation invariant form (Sec. 4.2, Algorithm 2), device buffers.
 * For sigma = -2, -1.5, .., 2 and theta = k pi/4 (k = 0..7) the method runs on
 * image 1 downsized by sigma1 = max(1, 2^sigma) against image 2 downsized by
 * sigma2 = max(1, 2^-sigma) and rotated by -theta.  A warped image lies on the
 * bounding box of the scaled, rotated image (sizes rounded to the nearest
 * integer), sampled bilinearly about the image centres, zero outside.  Every
 * atomic correspondence of every run (Eq. 15) is rectified to the input pair
 * (sigma1 p, sigma2 R_theta p' about the image centres, rounded to the
 * nearest pixel; p's atomic patch of I is the 4x4 cell holding that pixel)
 * and reduced into BestAt / BestAt' of the input pair; one reciprocal
 * verification (Eq. 16) then writes the matches as dm_match does: up to
 * `capacity` in atomic-patch order of image 1, *d_count (device int) the
 * number found.  Transforms that leave an image below 4 pixels, or with no
 * aggregation level, are skipped; a transform whose warped pair needs
 * 64-bit merge keys (the 45-degree canvases are the largest) gets them
 * (dm_set_merge_keys).  The precision and parameters are the context's.  The runs are
 * independent (their reductions are order-independent), so they are spread
 * over the context's concurrent lanes (dm_set_batch_lanes; longest run first,
 * each to the least loaded lane) that fork from and join back into `stream`;
 * the result does not depend on the number of lanes.  No host
 * synchronisation.  Status words of all runs are OR-ed into the header at
 * offset 0 of d_ws (dm_read_status; reached[] sums the runs).  d_ws is
 * 256-byte aligned and >= *bytes of dm_invariant_workspace_bytes (the size for
 * the context's lanes); a smaller workspace holding at least one lane's
 * region runs on fewer lanes, each lane's region reused by its runs in turn. */
dm_status dm_invariant_workspace_bytes(dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* bytes);
dm_status dm_match_invariant(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                             void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count,
                             void* stream);

/* Synchronise `stream` and read the header at offset 0 of a pyramid,
 * backtracking, dm_match or dm_match_invariant workspace: *status = DM_DEV_* bits (0 = fine;
 * DM_DEV_TIMEOUT if a bounded device-side wait of the pyramid step gave up);
 * reached[l] (l = 0..n_reached-1, may be NULL) = number of distinct merged
 * tuples at level l during the last backtracking (level 0: atomic tuples
 * before merging by pixel, i.e. arrivals). */
dm_status dm_read_status(dm_ctx* ctx, const void* d_ws, int* status, long long* reached, int n_reached,
                         void* stream);

/* Fault injection (no counterpart in the paper): test hooks that drive the
 * library's failure paths on the host or through bounded device waits, never
 * through a GPU fault.  Each hook stays armed until it fires or is reset.
 *   DM_FAULT_NONE      reset every hook of ctx and the process-wide one.
 *   DM_FAULT_LAUNCH    the arg-th next launch site of ctx (level-0
 *                      correlation, pyramid levels, backtracking of
 *                      dm_correlate_pyramid, dm_backtrack and dm_match) reports a
 *                      launch failure: the call returns DM_ECUDA with a message
 *                      naming the stage and "injected"; the stages before it
 *                      have been queued, the rest is not; later calls run
 *                      normally.  arg = 0: off.
 *   DM_FAULT_CAPACITY  the merge tables of dm_backtrack and dm_match hold at
 *                      most arg slots per level (rounded up to a multiple of
 *                      64): a pair with more merged tuples sets
 *                      DM_DEV_FRONTIER_OVERFLOW (dm_read_status) and returns
 *                      the matches of the tuples that fitted.  arg = 0: off.
 *   DM_FAULT_WAIT      every CTA of the level kernel (levels 1..L-1) first
 *                      waits arg clock cycles on a barrier nothing completes;
 *                      the bounded wait runs out, the CTA waits for the loads
 *                      it has started and exits, and dm_read_status on the
 *                      pyramid (or dm_match) workspace reports DM_DEV_TIMEOUT;
 *                      the pyramid's contents are then undefined.  arg = 0: off.
 *   DM_FAULT_ALLOC     process-wide (ctx may be NULL): the arg-th next resource
 *                      creation (dm_create's context, dm_timing_start's events)
 *                      fails with DM_ENOMEM and leaves nothing behind.
 * Not covered: a run-out of the tensor-core level-0 kernel's waits (its abort
 * path does not wait for the copies and MMAs already issued). */
#define DM_FAULT_NONE 0
#define DM_FAULT_LAUNCH 1
#define DM_FAULT_CAPACITY 2
#define DM_FAULT_WAIT 3
#define DM_FAULT_ALLOC 4
dm_status dm_inject_fault(dm_ctx* ctx, int kind, long long arg);

/* Differentiable form (the paper defines no loss; this one is the sum of the top-level maxima).
 * loss = sum over the existing top-level patches p of max_q C_L(p, q) (first
 * maximum), for the pyramid `pyr` built by dm_correlate_pyramid from d_desc1 /
 * d_desc2 (which must be unchanged).  Writes *d_loss (device float; summed in
 * double over patches in patch order), d_parts[p] (device, optional: the
 * per-patch maxima, [n_patch]) and, unless d_g1 or d_g2 is NULL, the
 * gradients d loss / d desc1 ([H1][W1][9]) and d loss / d desc2 ([H2][W2][9]).
 * The backward follows the forward exactly: through the power (Eq. 11), the
 * shifted average (Eq. 12), the max-pooling argmax saved by the forward
 * (Eq. 9) and the level-0 correlation (Eq. 3-4), whose values at the argmax
 * positions are recomputed instead of stored; only the gradient's support is
 * visited, level by level, and both level-0 products are gathers over the
 * argmax positions with a nonzero gradient.  All sums have a fixed order: the
 * gradient is deterministic.  d_ws >= dm_grad_workspace_bytes, any contents
 * (the call clears what it reads).  Both calls return DM_EUNSUPPORTED where a
 * level's support could exceed 2^32 entries (far beyond any size whose
 * workspace fits a GPU). */
dm_status dm_grad_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* bytes);
dm_status dm_loss_grad(dm_ctx* ctx, const dm_pyramid* pyr, const float* d_desc1, const float* d_desc2, void* d_ws,
                       size_t ws_bytes, float* d_loss, float* d_parts, float* d_g1, float* d_g2, void* stream);

/* One image pair of a batch (device buffers, as for dm_match). */
/* Width of the backtracking's merge keys (Sec. 3.3 "Merging correspondences":
 * tuples equal in (level, patch, position) are merged).  The key of a tuple
 * of level l is patch * |domain of l| + position; bits = 0 (default) takes
 * 32-bit keys in 8-byte table slots where every level's keys fit 32 bits and
 * 64-bit keys in 16-byte slots elsewhere (e.g. images of about 1024 x 512 and
 * more, and the rotated canvases of dm_match_invariant); bits = 64 takes
 * 64-bit keys at every size (the results are the same; used to test the wide
 * form on small pairs).  It applies to the calls made afterwards, workspace
 * queries included (64-bit keys double the tables' bytes): set it before
 * sizing workspaces.  DM* (dm_match_star, dm_backtrack_star) keeps 32-bit keys
 * and returns DM_EUNSUPPORTED for sizes that need 64.  DM_EINVAL for other
 * values of bits. */
dm_status dm_set_merge_keys(dm_ctx* ctx, int bits);

typedef struct {
    const float* d_img1;
    int W1, H1;
    const float* d_img2;
    int W2, H2;
    dm_match_t* d_out;
    int capacity;
    int* d_count;
} dm_pair;

/* Batched form.  Matches n pairs of possibly different sizes, with the
 * results of dm_match pair by pair.  The pairs run in waves of up to W pairs
 * (dm_set_batch_wave, 1 by default; dm_autotune_batch picks W and the number
 * of lanes for a batch and a workspace): within a wave every step of the method
 * is one launch for all of its pairs -- the descriptor passes, the operand
 * packing, one persistent level-0 kernel whose CTAs drain the work units of
 * every pair of the wave in turn, one launch per kernel and level of the
 * pyramid, one per step of the backtracking, one reciprocal verification --
 * each kernel taking the wave's per-pair arguments in its parameters and
 * mapping its blocks or work units onto (pair, unit), so that the small and
 * latency-bound steps of all pairs (the top levels, the backtracking) fill
 * the GPU together.  Waves run on the context's concurrent lanes (internal
 * streams; 2 by default, dm_set_batch_lanes): wave i on lane i % lanes.  Each
 * pair of a wave has its own slice of d_ws (pair j of the wave on lane k in
 * slice k W + j, at offset (k W + j) lane_bytes, lane_bytes = the largest
 * match_bytes over the pairs rounded up to 256); a smaller d_ws (at least
 * lane_bytes) runs narrower waves, then fewer lanes.  With W = 1 each pair
 * runs its own launches, pair k on lane k % lanes, so that the latency-bound
 * phases of one pair overlap the compute of another.  The lanes fork from
 * and join back into `stream` with events: all of the work is ordered after
 * what was already on `stream`, and work queued on `stream` later waits for
 * every pair.  dm_batch_workspace_bytes gives the slices of the configured
 * waves and lanes (W' K' lane_bytes, W' = min(W, n), K' = min(lanes, number
 * of waves)).  Nothing synchronises with the host, so the whole batch can be
 * captured in a CUDA graph and replayed (make one uncaptured call first so
 * that one-time per-device set-up does not happen inside the capture); the
 * per-pair arguments of the cross-pair launches are kernel parameters, which
 * the graph keeps.  Arguments of every pair are checked before anything is
 * launched.  Each pair's device status word is in the header of its slice
 * (dm_read_status on the slice reads the last pair that ran there). */
dm_status dm_batch_workspace_bytes(const dm_ctx* ctx, int n, const dm_pair* pairs, size_t* bytes);
dm_status dm_match_batch(dm_ctx* ctx, int n, const dm_pair* pairs, void* d_ws, size_t ws_bytes, void* stream);
/* One image pair of a host-buffer batch: images and outputs in host memory. */
typedef struct {
    const float* h_img1;
    int W1, H1;
    const float* h_img2;
    int W2, H2;
    dm_match_t* h_out;    /* first min(capacity, number of atomic patches) rows are written */
    int capacity;
    int* h_count;         /* number of matches (may exceed capacity: then only capacity rows) */
} dm_pair_host;

/* Batched form with host buffers (the whole chain as one call from host
 * memory: no counterpart in the paper).  As dm_match_batch, but every pair's
 * images are copied from host memory into its workspace slice, and its
 * matches and count copied back to host memory, inside its lane (before and
 * after its wave): the copies of one wave overlap the compute of the waves in
 * the other lanes.  Everything is
 * asynchronous on the lanes and `stream`; the host buffers must stay valid,
 * and the results are there, once `stream` has completed.  With page-locked
 * host buffers the copies are truly asynchronous and the whole call can be
 * captured in a CUDA graph (make one uncaptured call first); with pageable
 * buffers the copies are staged synchronously by the CUDA runtime and the call
 * cannot be captured.  A count above the capacity is reported only through
 * *h_count.  dm_batch_host_workspace_bytes gives the slices of the configured
 * waves and lanes as for dm_match_batch (lane_bytes = the largest match_bytes
 * over the pairs). */
dm_status dm_batch_host_workspace_bytes(const dm_ctx* ctx, int n, const dm_pair_host* pairs, size_t* bytes);
dm_status dm_match_batch_host(dm_ctx* ctx, int n, const dm_pair_host* pairs, void* d_ws, size_t ws_bytes, void* stream);

/* Number of concurrent lanes of dm_match_batch and dm_match_invariant, 1..4
 * (1: one wave, pair or transform after the other on `stream`). */
dm_status dm_set_batch_lanes(dm_ctx* ctx, int lanes);

/* Pairs per wave of dm_match_batch and dm_match_batch_host, 1..8 (1, the
 * default: every pair with its own launches). */
dm_status dm_set_batch_wave(dm_ctx* ctx, int pairs);

/* Autotuner of the batch shape: runs dm_match_batch on these pairs (once
 * untimed, then twice timed with CUDA events on `stream`, per candidate) for every wave width W in
 * {1, 2, 3, 4, 6, 8} and lanes K in 1..4 with W K slices of lane_bytes within
 * ws_bytes (and W <= n, K <= the number of waves), and keeps the fastest
 * (a candidate must beat the best so far by 2 %) as the context's wave width
 * and lanes; then, in that shape, it times the backtracking expansions at 4,
 * 8 and 16 CTAs per SM for all the batch's pair sizes together (concurrent
 * lanes share the SMs) and keeps the fastest in their launch shapes (or each
 * size's own).  chosen (may be NULL) receives {W, K}.  Synchronises with the host
 * (not capturable); the pairs' outputs hold the matches of the last run.
 * DM_ENOMEM if ws_bytes is below one lane_bytes.  Measured at 1024 x 436 (8
 * BF16 pairs, one graph): W = 1 on 2 lanes 61.6 pairs/s, waves of 2 on 2
 * lanes 60.1, W = 1 on 3 lanes 58.1, waves of 4 on one lane 57.9, W = 1 on
 * one lane 57.6 -- there one pair's kernels already fill the GPU and two
 * lanes overlap one pair's latency-bound steps with another's level 0. */
dm_status dm_autotune_batch(dm_ctx* ctx, int n, const dm_pair* pairs, void* d_ws, size_t ws_bytes, int* chosen,
                            void* stream);

/* Autotuner of the batched form.  Runs the launch-shape candidates of three
 * kernels on the given pair and keeps, for pairs of exactly these sizes in
 * this context, the fastest of each:
 *   chosen[0]  M-tiles (128 patches each) per work unit of the tensor-core
 *              level-0 kernel (the work unit is one N-tile x that many
 *              M-tiles; candidates split the patches into 1, 2, 3, 4, 6 or 8
 *              chunks; unused by DM_FP32);
 *   chosen[1]  level kernel: pooled rows per CTA tile of the tiled kernel (16,
 *              8 or 4, on 8, 4 or 2 warps), or 0 for the row-streaming kernel
 *              (one warp per patch and 31-column strip, no shared memory);
 *              levels whose stored maps are at most 16 columns wide always
 *              take the latter;
 *   chosen[2]  CTAs per SM of the backtracking expansion kernels (2..32);
 *   chosen[3]  child-window columns in the level kernel's ring (3 or 2).
 * Every candidate computes identical results; only the time differs.  Each
 * candidate runs three times (after one untimed run of the default), timed
 * with CUDA events, best of three; a candidate replaces the current choice
 * only when it is at least 3% faster.  Later
 * dm_correlate_pyramid / dm_match / dm_match_batch calls on pairs of these
 * sizes use the choice.  d_img1, d_img2, d_ws as for dm_match (d_ws is used as
 * scratch).  Synchronises `stream` (cannot be captured: tune before capturing
 * a graph).  chosen: 4 ints out, or NULL.  The paper has no counterpart. */
dm_status dm_autotune(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                      void* d_ws, size_t ws_bytes, int* chosen, void* stream);
/* The launch shapes used for pairs of these sizes (until dm_autotune has run
 * on them the defaults: all M-tiles in one work unit -- half of them for
 * DM_FP8_E4M3 --, 8, 8, 2): 4 ints as for dm_autotune. */
dm_status dm_tuned_config(dm_ctx* ctx, int W1, int H1, int W2, int H2, int* chosen);
/* Set the launch shapes for pairs of these sizes (e.g. a choice saved from an
 * earlier dm_autotune): chosen[0] >= 1, chosen[1] in {0, 4, 8, 16}, chosen[2] in
 * 1..64, chosen[3] in {2, 3}; DM_EINVAL otherwise. */
dm_status dm_set_tuned_config(dm_ctx* ctx, int W1, int H1, int W2, int H2, const int* chosen);

/* Backtracking without any caller workspace.
 * No counterpart in the paper: this entry point exists for callers that cannot
 * allocate device memory or hand the library a workspace -- plug-ins inside a
 * host application that owns all device memory and forbids allocations after
 * start-up, or latency-critical loops that must never call cudaMalloc (it can
 * synchronise the device).  It does what dm_backtrack does, with the same
 * kernels and results, but its scratch (merge tables, BestAt /
 * BestAt' keys, status header) is a fixed device array of
 * DM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  The caller still passes the pyramid
 * (input) and d_out / d_count (outputs), as for dm_backtrack.
 *   - Pairs whose backtracking scratch (backtrack_bytes of dm_workspace_bytes)
 *     exceeds DM_NOALLOC_SCRATCH_BYTES are refused with DM_ENOMEM and a message
 *     (32 MiB holds pairs up to about 160 x 120 pixels).
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.  Its first
 *     call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     and caches it; make that first call before any stream capture.  Under
 *     CUDA's lazy module loading (the default) that first look-up is also when
 *     the driver loads this part of the library and reserves the array, which
 *     can synchronise the device and fails (DM_ECUDA) if the application has
 *     already taken all device memory: make the first call at start-up, before
 *     the application claims the rest of the memory.  A context whose device
 *     cannot be made current gets DM_ECUDA before anything is looked up.
 *   - Every call uses the same array and leaves its contents behind; each call
 *     clears what must start empty.  Calls that overlap on the GPU (other
 *     streams, other threads) race on the array: serialise them.
 *   - The device status word is not readable through dm_read_status; an output
 *     overflow still shows as *d_count > capacity. */
#define DM_NOALLOC_SCRATCH_BYTES (32u << 20)
dm_status dm_backtrack_noalloc(dm_ctx* ctx, const dm_pyramid* pyr, dm_match_t* d_out, int capacity, int* d_count,
                               void* stream);

/* Stage timing (tracing).  After dm_timing_start(ctx, max_calls), each of the
 * next max_calls dm_match calls records CUDA events on its stream at the stage
 * boundaries: descriptors | level-0 correlation | levels >= 1 | backtracking.
 * dm_timing_read() waits for the last recorded event and returns, summed over
 * the recorded calls, the milliseconds of each stage (stage_ms[DM_NSTAGES]),
 * the number of calls recorded and the number of kernels the library launched
 * during them.  Events are created by dm_timing_start (no device memory). */
#define DM_NSTAGES 4
dm_status dm_timing_start(dm_ctx* ctx, int max_calls);
dm_status dm_timing_read(dm_ctx* ctx, double* stage_ms, int* n_calls, long long* n_launches);

#ifdef __cplusplus
}
#endif
#endif /* DM_H */
