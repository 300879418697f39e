/*
 * gsparc.h — C ABI of the GB300 (sm_103a) equirectangular Gaussian-splatting
 * library for RF spectra (the GSpaRC hot path).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status (GSPARC_OK or a negative code);
 *     no C++ exception crosses this boundary.
 *   - Every pointer argument named like a tensor is DEVICE memory owned by the
 *     caller, unless the comment says host.  The library never allocates
 *     device memory; scratch space comes from a caller-provided workspace
 *     whose size a *_workspace query returns.  One exception:
 *     gsparc_bin_sort_noalloc keeps its scratch in a fixed array of the
 *     library's own device memory (see its comment).
 *   - Every call takes a CUDA stream (cudaStream_t passed as void*, NULL for
 *     the legacy default stream), only enqueues work on it and returns without
 *     synchronising.  Argument errors are detected on the host before anything
 *     is enqueued.  Conditions only the device can see (a pair list longer
 *     than its capacity, an expired bounded wait) are written to a
 *     caller-provided device int32 status word; gsparc_check() reads it.
 *   - All float tensors are row-major FP32 unless stated otherwise; complex
 *     values are interleaved (re, im) FP32 pairs.
 *   - Gradient entry points (*_bwd) ACCUMULATE (+=) into their gradient
 *     outputs; the caller zeroes them first.
 *
 * Notation follows the paper (arxiv 2511.22793): means mu, covariance
 * Sigma = R S S^T R^T, opacity sigma, complex emission s, receiver-centric
 * coordinates x' = V (mu - x_rx), equirectangular pixel (p_x, p_y).
 */
#ifndef GSPARC_H
#define GSPARC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GSPARC_OK 0
#define GSPARC_ERR_INVALID (-1)   /* bad argument (detected on the host)          */
#define GSPARC_ERR_WORKSPACE (-2) /* workspace smaller than the query returned    */
#define GSPARC_ERR_CUDA (-3)      /* a CUDA runtime call or launch failed         */
#define GSPARC_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up           */
#define GSPARC_ERR_CAPACITY (-5)  /* more pairs (or densified rows) than capacity */
#define GSPARC_ERR_TOO_LARGE (-6) /* sizes above a fixed-scratch entry point's cap */
#define GSPARC_ERR_INPUT (-7)     /* the device found an input out of its domain     */

/* ---- fixed sizes ------------------------------------------------------- */
#define GSPARC_TILE 16       /* pixels per tile side                              */
#define GSPARC_LATENT 16     /* per-Gaussian latent width                         */
#define GSPARC_MLP_IN 20     /* network input: tx (3), latent (16), log d (1)     */
#define GSPARC_PROJ_STRIDE 8 /* floats per projection record                      */

/* Arithmetic of the attribute network (gsparc_attr_mlp). */
#define GSPARC_FP32 0   /* FP32 on CUDA cores                                        */
#define GSPARC_BF16 1   /* hidden layer on tensor cores, BF16 operands, FP32 accum.   */
#define GSPARC_BF16X2 2 /* as BF16 with each activation split into two BF16 terms    */

/*
 * Receiver view and hemisphere grid (Sec. 4.2, "Directional Projection and
 * Splatting"): x' = V (mu - rx); H rows of elevation (row 0 at the horizon,
 * row H-1 at the zenith, 90/H degrees each), W columns of azimuth (column W/2
 * looks along +z', 360/W degrees each).  Gaussians closer than near_dist to
 * the receiver are culled.  Host struct, passed by pointer.
 */
typedef struct gsparc_view {
    int32_t H, W;
    float rx[3];
    float V[9]; /* row-major 3x3, rotation world -> receiver frame */
    float near_dist;
} gsparc_view;

/*
 * Subcarriers (Sec. 3.1 channel model; Sec. 5 multi-subcarrier CSI):
 * f_k = f_c + (k - floor(K/2)) df, k = 0..K-1.  Host struct.
 */
typedef struct gsparc_band {
    int32_t K;
    int32_t reserved;
    double f_c, df; /* Hz */
} gsparc_band;

/*
 * Attribute network shared by all Gaussians (Eq. 1): input
 * h0 = [tx (3), latent (16), log d (1)], two ReLU hidden layers of width
 * `hidden` (8, 16, 32 or 64), three outputs.  Weights are input-major device
 * FP32 arrays: W1 [20, hidden], W2 [hidden, hidden], W3 [hidden, 3].
 * Host struct holding device pointers.
 */
typedef struct gsparc_mlp {
    int32_t hidden;
    int32_t reserved;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
} gsparc_mlp;

/* Gradient buffers of the network, same shapes as gsparc_mlp (device). */
typedef struct gsparc_mlp_grad {
    float *W1, *b1, *W2, *b2, *W3, *b3;
} gsparc_mlp_grad;

/* Number of 16x16 tiles covering the view: ceil(W/16) * ceil(H/16). */
int32_t gsparc_num_tiles(const gsparc_view* view);

/*
 * Project N Gaussians onto the equirectangular hemisphere (Sec. 4.2: view
 * transform, map p_x = (atan2(x', z')/pi + 1) W/2, p_y = 2 asin(y'/|x'|) H/pi,
 * and Sigma' = J V Sigma V^T J^T; Algorithm 1 CullGaussians / TransformToView
 * / ProjectGaussians).  Sigma = R(q) diag(exp(2 log_scales)) R(q)^T (Sec. 3.2).
 *   means [N,3], log_scales [N,3], quats [N,4] as (w, x, y, z), any norm > 0.
 *   proj [N,8] out: (p_x, p_y, ext_x, ext_y, c_xx, c_xy, c_yy, r), where c is
 *   the conic (Sigma' + 0.3 I)^-1, ext the footprint half extents
 *   sqrt(2 ln 255 * diag(Sigma' + 0.3 I)) in pixels and r = |x'|.  Culled
 *   Gaussians (r < near_dist) get ext_x = ext_y = -1.
 *   d_status [1] (device, may be NULL): set to GSPARC_ERR_INPUT when a
 *   Gaussian has a non-finite mean or log-scale or a zero quaternion; such a
 *   Gaussian is culled (ext = -1) and gsparc_project_bwd passes it no gradient.
 * Errors: GSPARC_ERR_INVALID for N < 0, a null pointer with N > 0 or a
 * non-positive H or W.
 */
int gsparc_project(const gsparc_view* view, int32_t N, const float* means, const float* log_scales,
                   const float* quats, float* proj, int32_t* d_status, void* stream);

/*
 * Gradient of gsparc_project (Sec. 4.2 map and Sigma'; Algorithm 1 Backprop).
 * d_proj [N,8] holds dL/d(p_x, p_y, -, -, c_xx, c_xy, c_yy, -) (slots 2, 3, 7
 * are ignored).  Accumulates into d_means [N,3] (atomically: it may run
 * concurrently with gsparc_attr_mlp_bwd(_tc), which also adds into d_means),
 * d_log_scales [N,3], d_quats [N,4].
 */
int gsparc_project_bwd(const gsparc_view* view, int32_t N, const float* means,
                       const float* log_scales, const float* quats, const float* d_proj,
                       float* d_means, float* d_log_scales, float* d_quats, void* stream);

/*
 * Bytes of workspace gsparc_bin_sort needs for N Gaussians and room for
 * pair_capacity (Gaussian, tile) pairs.  *ws_bytes is a host pointer.
 */
int gsparc_bin_sort_workspace(const gsparc_view* view, int32_t N, int64_t pair_capacity,
                              size_t* ws_bytes);

/*
 * Tile binning and directional sorting (Algorithm 1 IntersectGaussians and
 * its depth sort step, depth = distance to the receiver; Sec. 1 "directional
 * sorting").  For every Gaussian, the 16x16 tiles its footprint box touches
 * (azimuth wrapping at +-pi) each get one (Gaussian, tile) pair; every tile's
 * list is ordered by (r, index).  The pairs are counted per tile, emitted into
 * per-tile buckets as the unique 64-bit keys (bits(r) << 32) | index, and
 * each bucket is sorted by its own thread block: up to 24576 pairs in shared
 * memory, by a distribution sort over 8192 depth sub-buckets (each key ranked
 * against the few keys of its sub-bucket); a larger bucket by the same sort
 * over 16384 sub-buckets, either cut into slices of about 12288 pairs sorted
 * in shared memory by blocks of their own (when there are fewer tiles than
 * SMs) or whole with its keys scattered in the workspace; an LSD radix sort
 * (8-bit digits, only the bytes that vary in the bucket, in the workspace)
 * when the depths are too concentrated for the sub-buckets.
 *   proj [N,8]: records from gsparc_project (only p, ext and r are read).
 *   ws: device workspace of ws_bytes >= gsparc_bin_sort_workspace().
 *   sorted_ids [pair_capacity] out: Gaussian id of each sorted pair.
 *   sorted_keys [pair_capacity] out, may be NULL: (tile_id << 32) | bits(r)
 *   of each sorted pair.
 *   tile_ranges [num_tiles, 2] out: [start, end) of each tile in sorted_ids
 *   ([0, 0) for an empty tile).
 *   n_pairs [1] out (device): number of pairs.
 *   d_status [1] (device): set to GSPARC_ERR_CAPACITY if the pairs exceed
 *   pair_capacity; the tiles whose lists end at or below pair_capacity (in
 *   tile order) are then complete and sorted, every later tile is [0, 0).
 * Pair capacity must be below 2^31.
 */
int gsparc_bin_sort(const gsparc_view* view, int32_t N, const float* proj, int64_t pair_capacity,
                    void* ws, size_t ws_bytes, uint32_t* sorted_ids, uint64_t* sorted_keys,
                    uint32_t* tile_ranges, uint32_t* n_pairs, int32_t* d_status, void* stream);

/*
 * gsparc_bin_sort without a workspace: the same binning and sort, bit for bit,
 * for callers that cannot allocate device memory.  (The paper has no
 * counterpart; this is a deployment variant of the call above.)  Some callers
 * may not call cudaMalloc at all: a real-time loop that must not take the
 * implicit device-wide synchronisation and unbounded latency of an allocation
 * after start-up, or a plugin whose host hands it buffers but no allocator.
 * They still pass every input and output; the scratch space (tile counters,
 * bucket cursors, the two key buffers) is a fixed 9 MiB array in the
 * library's own device memory, which every GPU that loads the library holds
 * until the process exits.
 *   Limits: N <= GSPARC_NOALLOC_MAX_N and pair_capacity <=
 *   GSPARC_NOALLOC_MAX_PAIRS; larger sizes return GSPARC_ERR_TOO_LARGE before
 *   anything is enqueued.  Other arguments and errors as gsparc_bin_sort.
 *   The first call on each device looks up that device's address of the
 *   array (with the device current); make that first call before any stream
 *   capture.  If that lookup fails (GSPARC_ERR_CUDA, e.g. a pending error of
 *   an earlier launch), nothing is cached and the next call tries again.
 *   The call allocates nothing.
 *   Every call on a device shares the one array and it keeps what the last
 *   call left there: the call clears what must start at zero itself, but two
 *   calls whose work overlaps on the GPU (different streams, no ordering
 *   between them) race on the array and both results are undefined.
 */
#define GSPARC_NOALLOC_MAX_N 65536
#define GSPARC_NOALLOC_MAX_PAIRS 524288
int gsparc_bin_sort_noalloc(const gsparc_view* view, int32_t N, const float* proj,
                            int64_t pair_capacity, uint32_t* sorted_ids, uint64_t* sorted_keys,
                            uint32_t* tile_ranges, uint32_t* n_pairs, int32_t* d_status,
                            void* stream);

/*
 * Attribute network for B transmitter positions (Eq. 1 with the 1/d of the
 * Sec. 4.2 compositing rule; query = transmitter, receiver fixed).
 *   d_i = max(|mu_i - tx_b|, 0.01); o = MLP([tx_b, latent_i, ln d_i]);
 *   attr[b,i] = (a, phi0, sigma, L) with a = sigmoid(o_0 - ln d_i)/d_i,
 *   phi0 = o_1, sigma = sigmoid(opacity_logit_i + o_2),
 *   L = d_i + |mu_i - rx| (path length, metres).
 *   tx [B,3] device; rx [3] HOST; means [N,3]; opacity_logit [N]; latent [N,16];
 *   attr [B,N,4] out.  precision: GSPARC_FP32, GSPARC_BF16 or GSPARC_BF16X2.
 *   hidden (may be NULL; GSPARC_FP32 only, else GSPARC_ERR_INVALID) out: the
 *   post-ReLU activations for gsparc_attr_mlp_bwd, feature-major
 *   [2 * mlp->hidden][ld], ld = B*N rounded up to a multiple of 4, row
 *   b*N + i: h1 in the first mlp->hidden feature rows, h2 in the next;
 *   16-byte aligned.  The ld - B*N padding columns are not written.
 */
int gsparc_attr_mlp(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                    const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                    int32_t precision, float* attr, float* hidden, void* stream);

/*
 * Gradient of gsparc_attr_mlp in FP32 (Algorithm 1 Backprop through the
 * network).  d_attr [B,N,4] holds dL/d(a, phi0, sigma, L).  Accumulates into
 * d_means [N,3], d_opacity_logit [N], d_latent [N,16] and every buffer of
 * *grads.  hidden: the activations an FP32 gsparc_attr_mlp call of the same
 * inputs stored (layout there; 16-byte aligned), read in place of
 * recomputing them; NULL recomputes them.
 */
int gsparc_attr_mlp_bwd(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                        const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                        const float* d_attr, float* d_means, float* d_opacity_logit,
                        float* d_latent, const gsparc_mlp_grad* grads, const float* hidden,
                        void* stream);

/*
 * gsparc_attr_mlp_bwd with the network's matrix products on the tensor cores
 * (Algorithm 1 Backprop through the network; same arguments plus precision,
 * same accumulation into the outputs).  Per tile of 128 rows the forward
 * recompute h0 W1, h1 W2 and the input gradients du2 W2^T, du1 W1^T are
 * tcgen05 products, and the weight and bias gradients are one product over
 * the rows, [h0 | h1 | h2 | 1]^T [du1 | du2 | dL/do], accumulated in tensor
 * memory over all the tiles of a thread block.  Operands are split into two
 * BF16 terms (three products, ~16-bit operands), accumulation is FP32.
 *   precision: GSPARC_BF16X2 (the only form).  mlp->hidden: 16 or 32; other
 *   widths return GSPARC_ERR_INVALID (use gsparc_attr_mlp_bwd).
 *   An expired wait on the tensor cores writes NaN into grads->b3[0].
 */
int gsparc_attr_mlp_bwd_tc(int32_t N, int32_t B, const float* tx, const float* rx, const float* means,
                           const float* opacity_logit, const float* latent, const gsparc_mlp* mlp,
                           int32_t precision, const float* d_attr, float* d_means,
                           float* d_opacity_logit, float* d_latent, const gsparc_mlp_grad* grads,
                           void* stream);

/*
 * Per-Gaussian emission network, the paper's own form of Eq. 1 (Sec. 4.1;
 * by the Sec. 4.2 implementation notes every Gaussian carries a network
 * R^3 -> R^2 with one hidden layer, 16 units in the paper, 8..64 in its Sec. 7
 * sweep).  For transmitter x = tx[b] and
 * Gaussian i with hidden width h:
 *   o = W2_i^T relu(W1_i^T x + b1_i) + b2_i,  d = max(|mu_i - x|, 0.01),
 *   s = sigmoid(o_0 - ln d) + j sigmoid(o_1 - ln d)   (element-wise, Eq. 1),
 *   attr[b,i] = (a, phi0, sigma, L) = (|s| / d, arg s, sigmoid(logit_i),
 *               d + |mu_i - rx|),
 * with |s| in place of |s| / d when inv_d is 0 (the 1/d term of the Sec. 4.2
 * compositing rule switched off, the Sec. 7 ablation), so that a e^{j phi0} =
 * s / d feeds the renderer unchanged.
 *   weights [N, stride] device, stride = gsparc_emission_stride(h): row i is
 *   W1 [3, h] (input-major), b1 [h], W2 [h, 2] (input-major), b2 [2], then
 *   padding to a multiple of 4 floats (ignored); 16-byte aligned.
 *   tx [B,3] device; rx [3] HOST; means [N,3]; opacity_logit [N];
 *   attr [B,N,4] out (16-byte aligned).  hidden in 1..64; N < 2^26 and
 *   N * B < 2^31 (GSPARC_ERR_INVALID otherwise).
 * One thread per Gaussian over every transmitter, the block's weight rows
 * staged in shared memory (the pass streams 4 * stride bytes per Gaussian).
 */
int32_t gsparc_emission_stride(int32_t hidden);
int gsparc_emission_fwd(int32_t N, int32_t B, int32_t hidden, const float* tx, const float* rx,
                        const float* means, const float* opacity_logit, const float* weights,
                        int32_t inv_d, float* attr, void* stream);

/*
 * Gradient of gsparc_emission_fwd for the upstream d_attr [B,N,4]
 * (dL/d(a, phi0, sigma, L)): ADDS into d_means [N,3] and d_opacity_logit [N]
 * (atomically, so another kernel may add into them concurrently) and into
 * d_weights [N, stride] (the padding untouched); summed over the B
 * transmitters.  The distance clamp passes no gradient; the ReLU's derivative
 * at 0 is 0.
 */
int gsparc_emission_bwd(int32_t N, int32_t B, int32_t hidden, const float* tx, const float* rx,
                        const float* means, const float* opacity_logit, const float* weights,
                        int32_t inv_d, const float* d_attr, float* d_means, float* d_opacity_logit,
                        float* d_weights, void* stream);

/*
 * Front-to-back compositing of complex contributions across subcarriers
 * (Sec. 4.2 compositing rule; Algorithm 1 inner loop): for every pixel u and
 * subcarrier k of every transmitter b,
 *   z[b,k,u] = sum_i T_i alpha_i a_i exp(j(phi0_i - 2 pi f_k L_i / c)),
 *   alpha_i = min(0.99, sigma_i exp(-q_i(u)/2)), T_i = prod_{j<i}(1 - alpha_j),
 * over the tile's list in (r, index) order, skipping q > 2 ln 255 or
 * alpha < 1/255 and stopping before T would fall below 1e-4.  T is carried
 * as log2 T in FP32.
 *   proj [N,8], tile_ranges [num_tiles,2], sorted_ids: from gsparc_bin_sort.
 *   attr [B,N,4]: from gsparc_attr_mlp.
 *   spectrum [B,K,H,W,2] out (complex, interleaved).
 *   final_logT [B,H,W] out, may be NULL: log2 of the transmittance left.
 *   n_contrib [B,H,W] out, may be NULL: 1 + position (within the tile list)
 *   of the last Gaussian composited, 0 if none.  gsparc_render_bwd needs both.
 *   n_used [B,H,W] out, may be NULL: number of Gaussians composited at the
 *   pixel (the algorithmic work per pixel and subcarrier).
 *   d_status [1] (device, may be NULL): set to GSPARC_ERR_INPUT when a tile
 *   list holds an id >= N (inconsistent inputs); that entry is skipped.
 */
int gsparc_render_fwd(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                      const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                      const float* attr, float* spectrum, float* final_logT, uint32_t* n_contrib,
                      uint32_t* n_used, int32_t* d_status, void* stream);

/*
 * gsparc_render_fwd with the complex L2 loss of gsparc_l2_loss fused into its
 * epilogue (the training step's loss, Algorithm 1; complex L2 in place of
 * Eq. 4), all arithmetic FP32 on the CUDA cores.  With count = B*K*H*W,
 *   loss [1] = mean |z - target|^2 (the call clears it first; blocks add
 *   partial sums atomically, so the last bits may differ from run to run),
 *   d_spectrum [B,K,H,W,2] out = 2 (z - target) / count, bit-identical to
 *   gsparc_l2_loss on the spectrum gsparc_render_fwd writes.
 * spectrum may be NULL (then it is never written).  s_tot may be NULL; else
 * [B, strips, H, W] out with strips = 1 for K <= 32 and ceil(K / 32) above:
 * s_tot[b,s,p] = sum over strip s's subcarriers of Re(conj(d_spectrum) z), the
 * input gsparc_render_bwd_balanced takes in place of the spectrum.  tile_walk
 * may be NULL; else [B, T] out: per (transmitter, tile) min(largest n_contrib
 * of its pixels, list length).  final_logT, n_contrib, n_used and d_status as
 * gsparc_render_fwd.
 */
int gsparc_render_fwd_l2(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                         const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                         const float* attr, const float* target, float* loss, float* d_spectrum,
                         float* spectrum, float* final_logT, uint32_t* n_contrib, uint32_t* n_used,
                         float* s_tot, uint32_t* tile_walk, int32_t* d_status, void* stream);

/*
 * gsparc_render_fwd with the subcarrier sum on the tensor cores (same
 * arguments, same outputs).  The per-pixel weights w_i = T_i alpha_i are taken
 * exactly as in gsparc_render_fwd (identical alpha, log2 T, cut-off and
 * termination decisions, hence identical final_logT, n_contrib and n_used);
 * the sum over the tile list of w_i s_ik (Sec. 4.2 compositing rule) runs as
 * tcgen05 matrix products over batches of 32 list entries, with w and s each
 * split into two BF16 terms (three products, ~16-bit operands) and FP32
 * accumulation in tensor memory.  Spectra agree with gsparc_render_fwd to
 * ~1e-5 relative.
 *   d_status [1] (device, may be NULL): GSPARC_ERR_INPUT as gsparc_render_fwd;
 *   GSPARC_ERR_TIMEOUT when a bounded wait of the kernel's pipeline expired
 *   (the affected strips of the spectrum are then NaN).  The kernel always
 *   lets its tensor-core products finish before it frees its tensor memory.
 */
int gsparc_render_fwd_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                         const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                         const float* attr, float* spectrum, float* final_logT,
                         uint32_t* n_contrib, uint32_t* n_used, int32_t* d_status, void* stream);

/*
 * Gradient of gsparc_render_fwd (Algorithm 1 Backprop through compositing and
 * splatting).  Walks each pixel's list back to front from n_contrib,
 * recovering T_i from final_logT by subtracting log2(1 - alpha_i), so no
 * per-pair state is stored.  d_spectrum [B,K,H,W,2] holds dL/dRe z, dL/dIm z.
 * Accumulates dL/d(a, phi0, sigma, L) into d_attr [B,N,4] and
 * dL/d(p_x, p_y, -, -, c_xx, c_xy, c_yy, -) into d_proj [N,8].
 * d_status [1] (device, may be NULL): GSPARC_ERR_INPUT as gsparc_render_fwd.
 */
int gsparc_render_bwd(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                      const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                      const float* attr, const float* final_logT, const uint32_t* n_contrib,
                      const float* d_spectrum, float* d_attr, float* d_proj, int32_t* d_status,
                      void* stream);

/*
 * gsparc_render_bwd with its three per-(pixel, Gaussian) subcarrier sums on the
 * tensor cores (same arguments, same outputs): Re and Im of
 * sum_k conj(dL/dz_k) e^{j psi_k} and the subcarrier-weighted Im sum that gives
 * dL/dL.  The upstream gradient of the strip is one operand, the Gaussians'
 * unit phasors the other, both split into two BF16 terms with FP32
 * accumulation in tensor memory; the back-to-front recursion (recovered T,
 * suffix sums, alpha and conic derivatives) runs on the CUDA cores exactly as
 * in gsparc_render_bwd.  Gradients agree with gsparc_render_bwd to ~1e-5.
 * The kernel is warp-specialised (producer warps build the phasor operand and
 * issue the products; the pixel warps consume them through mbarriers).  An
 * expired bounded wait leaves the gradients incomplete, adds NaN to
 * d_attr[b,0,0] of the affected transmitter and sets d_status [1] (device,
 * may be NULL) to GSPARC_ERR_TIMEOUT; GSPARC_ERR_INPUT as gsparc_render_fwd.
 * The kernel always lets its tensor-core products finish before it frees its
 * tensor memory.
 */
int gsparc_render_bwd_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                         const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                         const float* attr, const float* final_logT, const uint32_t* n_contrib,
                         const float* d_spectrum, float* d_attr, float* d_proj, int32_t* d_status,
                         void* stream);

/*
 * Bytes of device workspace gsparc_render_bwd_tc_balanced needs for B
 * transmitters of this view and band: 16 + 4 B T (rounded up to 16) +
 * 32 B T strips, T = tiles, strips as for s_tot.
 */
int gsparc_render_bwd_tc_workspace(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                   size_t* ws_bytes);

/*
 * gsparc_render_bwd_tc with its work scheduled over the SMs (same gradients
 * up to rounding order).  The cost of a (transmitter, tile, strip) is its
 * walk, the largest n_contrib among the tile's pixels, and varies by a
 * factor of two or more between tiles.  A first kernel takes every walk
 * and builds an ordered list of work items; a walk longer than split_min
 * batches of 16 entries is split into a front chunk [0, m) and a back
 * chunk [m, walk) (m = 16 floor(batches / 2)), run as independent blocks.
 * The back chunk walks back to front from the final state as
 * gsparc_render_bwd_tc does.  The front chunk walks front to back from
 * T = 1 (the forward's own recursion) and takes the suffix sum of entry i,
 * sum_{j>i} w_j Re(conj(g) s_j), as s_tot - sum_{j<=i} (Algorithm 1's
 * Backprop; the identity sum_j w_j s_j = z), so no state at m is needed.
 * Items are ordered by decreasing batch count: the block scheduler hands out
 * blocks in index order, so the SMs take the longest items first.
 *   spectrum [B,K,H,W,2] or NULL; s_tot [B,strips,H,W] (from
 *   gsparc_render_fwd_l2_tc) or NULL: the front chunks take s_tot when given,
 *   else form it from the spectrum and d_spectrum; with both NULL no walk is
 *   split (the items are still ordered).
 *   tile_walk [B, T] (from gsparc_render_fwd_l2_tc) or NULL: given, the
 *   schedule is one block that reads it; NULL, one block per tile first
 *   takes each walk from n_contrib.
 *   split_min: 0 selects the default (3 batches), a negative value disables
 *   splitting; walks are split only while B * T * strips <= 2 x SMs (with
 *   more units the ordering alone keeps the SMs busy).
 *   ws: device workspace of ws_bytes >= gsparc_render_bwd_tc_workspace(),
 *   16-byte aligned, whose first 16 bytes are zero before its first use
 *   (every call leaves them zero again); one call at a time per workspace.
 * Other arguments, outputs and the status word as gsparc_render_bwd_tc; the
 * front chunks' suffix is a difference of two sums, so its error is relative
 * to s_tot, not to the suffix (the gradients agree with gsparc_render_bwd_tc
 * to ~1e-5 relative L2).
 */
int gsparc_render_bwd_tc_balanced(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                                  const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                                  const float* attr, const float* spectrum, const float* s_tot,
                                  const uint32_t* tile_walk, const float* final_logT, const uint32_t* n_contrib,
                                  const float* d_spectrum, int32_t split_min, void* ws, size_t ws_bytes,
                                  float* d_attr, float* d_proj, int32_t* d_status, void* stream);

/*
 * Bytes of device workspace gsparc_render_bwd_balanced needs for B
 * transmitters of this view and band: 16 + 4 B T (rounded up to 16) +
 * 32 B T strips, T = tiles, strips as for the s_tot of gsparc_render_fwd_l2.
 */
int gsparc_render_bwd_workspace(const gsparc_view* view, const gsparc_band* band, int32_t B,
                                size_t* ws_bytes);

/*
 * gsparc_render_bwd with its work scheduled over the SMs, in FP32 on the CUDA
 * cores (same gradients up to rounding order).  The schedule is that of
 * gsparc_render_bwd_tc_balanced: every (transmitter, tile, strip of up to 32
 * subcarriers) walk, the largest n_contrib among the tile's pixels, becomes one
 * work item, or, when longer than split_min batches of 16 entries, a front
 * chunk [0, m) walked front to back from T = 1 with the suffix sum taken as
 * s_tot minus the prefix, and a back chunk [m, walk) walked back to front from
 * the final state; items run longest first.  Splitting is on while the
 * (transmitter, tile, strip) units are at most four times the SM count.
 *   spectrum [B,K,H,W,2] or NULL; s_tot (from gsparc_render_fwd_l2) or NULL:
 *   the front chunks take s_tot when given, else form it from the spectrum;
 *   with both NULL no walk is split.  tile_walk [B, T] or NULL as in
 *   gsparc_render_bwd_tc_balanced.  split_min: 0 the default (3), < 0 none.
 *   ws: gsparc_render_bwd_workspace() bytes, 16-byte aligned, its first 16
 *   bytes zero before first use (every call leaves them zero); one call at a
 *   time per workspace.
 * Other arguments, outputs and the status word as gsparc_render_bwd.
 */
int gsparc_render_bwd_balanced(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                               const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                               const float* attr, const float* spectrum, const float* s_tot,
                               const uint32_t* tile_walk, const float* final_logT, const uint32_t* n_contrib,
                               const float* d_spectrum, int32_t split_min, void* ws, size_t ws_bytes,
                               float* d_attr, float* d_proj, int32_t* d_status, void* stream);

/*
 * Complex L2 loss, the mean over `count` complex elements of |z - target|^2,
 * written to loss [1] (device; overwritten), and if d_z is not NULL its
 * gradient 2 (z - target) / count (overwritten).
 */
int gsparc_l2_loss(int64_t count, const float* z, const float* target, float* loss, float* d_z,
                   void* stream);

/*
 * CSI head (Sec. 4.2 "Rendered Spectrum", Eq. 2): the complex channel
 * estimate of each (transmitter, subcarrier) is the spatial mean of its
 * spectrum plane, csi[b,k] = scale * sum_p spectrum[b,k,p] (scale = 1/(H W)
 * for the mean).
 *   spectrum [B,K,P,2] (complex, interleaved; P = H*W pixels); csi [B,K,2]
 *   out (overwritten).  B*K < 65536.  Blocks add partial sums atomically:
 *   the result may differ in the last bits from run to run.
 */
int gsparc_csi_head(int32_t B, int32_t K, int64_t P, const float* spectrum, float scale, float* csi,
                    void* stream);

/*
 * Channel loss (Eq. 3, the squared error of the real and imaginary parts),
 * averaged over the B*K (transmitter, subcarrier) entries:
 *   loss [1] = mean |csi - target|^2 (overwritten); d_csi [B,K,2] out, may be
 *   NULL: 2 (csi - target) / (B K) (overwritten).
 */
int gsparc_csi_loss(int32_t B, int32_t K, const float* csi, const float* target, float* loss,
                    float* d_csi, void* stream);

/*
 * Gradient of gsparc_csi_head: d_spectrum[b,k,p] = scale * d_csi[b,k] at every
 * pixel p (overwritten).  d_csi [B,K,2]; d_spectrum [B,K,P,2].
 */
int gsparc_csi_head_bwd(int32_t B, int32_t K, int64_t P, const float* d_csi, float scale,
                        float* d_spectrum, void* stream);

/*
 * Magnitude-spectrum loss (Eq. 4): L = (1 - lambda) L1(|z|, y) + lambda (1 -
 * SSIM(|z|, y)), the paper's loss when the target is a magnitude spectrum
 * (lambda_1 = 0.2 in the paper).  L1 is the mean |x - y| over every
 * (transmitter, subcarrier, pixel), x = |z|; SSIM is taken per (transmitter,
 * subcarrier) plane with an 11 x 11 Gaussian window (sigma 1.5, normalised),
 * zero padding with the output the size of the plane, C1 = 0.01^2,
 * C2 = 0.03^2, as the mean of the SSIM map, averaged over planes.
 *   spectrum [B,K,H,W,2] (complex); target [B,K,H,W] (real magnitudes);
 *   loss [1] out (overwritten); d_spectrum [B,K,H,W,2] out (overwritten) or
 *   NULL: dL/dRe z, dL/dIm z = dL/dx z / |z|, 0 where z = 0 (and the L1
 *   term's derivative 0 where x = y).
 *   ws: device workspace of ws_bytes >= gsparc_spectrum_loss_workspace()
 *   (44 B per pixel and plane + 256), 16-byte aligned.
 * Separable filtering in four passes over whole maps (HBM-bound); sums
 * accumulate in double atomically, so the last bits of the loss may differ
 * between runs.
 */
int gsparc_spectrum_loss_workspace(int32_t B, int32_t K, int32_t H, int32_t W, size_t* ws_bytes);
int gsparc_spectrum_loss(int32_t B, int32_t K, int32_t H, int32_t W, const float* spectrum,
                         const float* target, float lambda, void* ws, size_t ws_bytes, float* loss,
                         float* d_spectrum, void* stream);

/*
 * gsparc_render_fwd_tc with the complex L2 loss of gsparc_l2_loss fused into its
 * epilogue (the training step's loss, Algorithm 1; complex L2 in place of
 * Eq. 4): with count = B*K*H*W,
 *   loss [1] = mean |z - target|^2 (the call clears it first; blocks add
 *   partial sums atomically, so the last bits may differ from run to run),
 *   d_spectrum [B,K,H,W,2] out = 2 (z - target) / count, bit-identical to
 *   gsparc_l2_loss on the spectrum gsparc_render_fwd_tc writes.
 * spectrum may be NULL (then it is never written: training needs only the
 * gradient); final_logT, n_contrib, n_used as gsparc_render_fwd.
 * s_tot may be NULL; else [B, strips, H, W] out, strips = ceil(K / 64) for
 * K > 64 and 1 otherwise: s_tot[b,s,p] = sum over the strip's subcarriers of
 * Re(conj(d_spectrum) z), the input gsparc_render_bwd_tc_balanced takes in
 * place of the spectrum (4 bytes per pixel and strip instead of 8 per
 * subcarrier).
 * tile_walk may be NULL; else [B, T] out (T = tiles): per (transmitter,
 * tile) the walk min(largest n_contrib of its pixels, list length), which
 * gsparc_render_bwd_tc_balanced takes in place of its own walk pass.
 * d_status as gsparc_render_fwd_tc (an expired wait makes the loss NaN).
 */
int gsparc_render_fwd_l2_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                            const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                            const float* attr, const float* target, float* loss, float* d_spectrum,
                            float* spectrum, float* final_logT, uint32_t* n_contrib, uint32_t* n_used,
                            float* s_tot, uint32_t* tile_walk, int32_t* d_status, void* stream);

/*
 * gsparc_render_fwd_tc with the CSI head fused into its epilogue: every
 * thread block sums its tile's pixels of each subcarrier and adds 1/(H W)
 * of it to csi [B,K,2] (overwritten: the call clears it first).  spectrum may
 * be NULL, and then the spectrum is never written (8 B per pixel, subcarrier
 * and transmitter saved) -- the form a CSI query at an unseen position needs.
 * final_logT, n_contrib, n_used as gsparc_render_fwd (each may be NULL).
 * Atomic partial sums: the last bits may differ from run to run.  d_status as
 * gsparc_render_fwd_tc (an expired wait makes the estimate NaN).
 */
int gsparc_render_csi_tc(const gsparc_view* view, const gsparc_band* band, int32_t B, int32_t N,
                         const float* proj, const uint32_t* tile_ranges, const uint32_t* sorted_ids,
                         const float* attr, float* csi, float* spectrum, float* final_logT,
                         uint32_t* n_contrib, uint32_t* n_used, int32_t* d_status, void* stream);

/*
 * Confidence-weighted objective (Eq. 5, Sec. 4.2 confidence-weighted
 * optimisation): a network g: R^3 -> R with one ReLU hidden layer maps each
 * sample's query position to the confidence C_b = 1 + exp(g(pos_b)) > 1, and
 * the objective is mean_b (C_b L_b - alpha ln C_b) (alpha = 0.3 and 32 hidden
 * units in the paper).  One call writes the objective, C and dObj/dL_b, and
 * accumulates the weight gradients.
 *   B >= 0 samples (B = 0: objective 0, nothing else written); hidden 1..32;
 *   pos [B,3], task_loss [B] in; weights: W1 [3,hidden] (input-major), b1
 *   [hidden], W2 [hidden], b2 [1] = 5 hidden + 1 floats; alpha >= 0;
 *   objective [1] out (overwritten); confidence [B] out, d_task_loss [B] out
 *   (C_b / B), both overwritten, may be NULL; d_weights [5 hidden + 1]
 *   accumulated (+=), may be NULL.
 * One block of 8 warps with a fixed summation order: results are the same
 * from run to run.
 */
int gsparc_confidence(int32_t B, int32_t hidden, const float* pos, const float* task_loss,
                      const float* weights, float alpha, float* confidence, float* objective,
                      float* d_task_loss, float* d_weights, void* stream);

/*
 * Adaptive density control (Algorithm 1, densification branch; Sec. 4.2
 * "Densification, Pruning, and Implementation").  The paper gives no
 * thresholds; the fields hold them (proposed values in brackets, 3D Gaussian
 * Splatting conventions where it has one).
 */
typedef struct gsparc_densify_params {
    float tau_grad;    /* mean ||dL/dmu|| at or above which a Gaussian grows [2e-4] */
    float clone_scale; /* eps * r_scene: a growing Gaussian whose largest per-axis
                          scale (m) is at most this is cloned, else split [0.01 * 5 sqrt 3] */
    float sigma_min;   /* opacity below which a Gaussian is pruned [0.005]           */
    float r_max;       /* footprint radius (px) above which a Gaussian is pruned [20] */
    int32_t n_split;   /* children of a split, 1..8 [2]                               */
} gsparc_densify_params;

/*
 * Statistic of the densification: every Gaussian whose projection record (as
 * written by gsparc_project: [N,8], ext_x and ext_y at offsets 2 and 3, -1 when
 * culled) has a footprint radius max(ext_x, ext_y) > 0 adds ||d_means[i]|| to
 * norm_sum[i] and 1 to count[i].
 *   proj [N,8], d_means [N,3] in; norm_sum [N] FP32 and count [N] u32
 *   accumulated (zero them after each densification).  N * 8 < 2^31.
 */
int gsparc_densify_accumulate(int32_t N, const float* proj, const float* d_means, float* norm_sum,
                              uint32_t* count, void* stream);

/* Workspace of gsparc_densify for N Gaussians: 4 B per 256 Gaussians, rounded up to 256 B. */
int gsparc_densify_workspace(int32_t N, size_t* ws_bytes);

/*
 * One densification: grow = count > 0 and norm_sum / count >= tau_grad;
 * a growing Gaussian with exp(max log-scale) <= clone_scale is cloned (an
 * exact copy), any other growing one is split into n_split children at
 * mu + R diag(exp(l)) xi[i, c] with log-scales l - ln(0.8 n_split), the rest
 * copied, the parent removed; then every output whose opacity sigmoid(logit)
 * is below sigma_min goes, and every Gaussian that existed before this call
 * whose footprint radius max(ext_x, ext_y) in proj exceeds r_max goes (clones
 * and children stay).  Outputs keep parent-index order, each parent's rows in
 * place: itself, then its clone; or its children in order.
 *   Inputs [N,...]: means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z),
 *   opacity_logit [N], payload [N,P] (per-Gaussian values copied along, e.g.
 *   latents or emission weights; may be NULL when P = 0), proj [N,8],
 *   norm_sum [N], count [N], xi [N, n_split, 3] standard-normal draws (row i
 *   serves Gaussian i if it splits).
 *   Outputs, `capacity` rows each, must not alias the inputs: out_means,
 *   out_log_scales, out_quats, out_opacity_logit, out_payload [capacity,P],
 *   out_parent [capacity] (the input index each row came from); n_out [1]
 *   (device u32) = the number of rows the densification produces.  Rows past
 *   the capacity are not written and the status word gets
 *   GSPARC_ERR_CAPACITY.  ws: gsparc_densify_workspace bytes, 4-byte aligned
 *   (GSPARC_ERR_WORKSPACE when smaller).
 * Three launches (count per block, one block scanning the block counts,
 * scatter); decisions in FP32; the result is the same from run to run.
 */
int gsparc_densify(int32_t N, int32_t P, const float* means, const float* log_scales, const float* quats,
                   const float* opacity_logit, const float* payload, const float* proj,
                   const float* norm_sum, const uint32_t* count, const float* xi,
                   const gsparc_densify_params* params, int32_t capacity, void* ws, size_t ws_bytes,
                   float* out_means, float* out_log_scales, float* out_quats, float* out_opacity_logit,
                   float* out_payload, uint32_t* out_parent, uint32_t* n_out, int32_t* d_status,
                   void* stream);

/*
 * Periodic opacity reset (Algorithm 1): sigma <- min(sigma, max_opacity) for
 * every Gaussian, on the logits: logit <- min(logit, ln(m / (1 - m))), in
 * place.  0 < max_opacity < 1 (0.01 in the paper).
 */
int gsparc_opacity_reset(int32_t N, float max_opacity, float* opacity_logit, void* stream);

/*
 * Adam step (Algorithm 1 "Adam"): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps), in place over
 * n FP32 elements.  step >= 1.
 */
int gsparc_adam(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float b1,
                float b2, float eps, int32_t step, void* stream);

/*
 * gsparc_adam over several parameter groups of one flat buffer in one launch
 * (Algorithm 1 "Adam" with the per-group learning rates of the paper's
 * hyperparameter table): group s covers elements [seg_end[s-1], seg_end[s])
 * (seg_end[-1] = 0) and takes learning rate seg_lr[s].  seg_end and seg_lr
 * are HOST arrays of n_seg (1..32) entries, seg_end non-decreasing with
 * seg_end[n_seg-1] = n; the same update and bias correction as gsparc_adam
 * otherwise.
 */
int gsparc_adam_segments(int64_t n, float* param, const float* grad, float* m, float* v, int32_t n_seg,
                         const int64_t* seg_end, const float* seg_lr, float b1, float b2, float eps,
                         int32_t step, void* stream);

/*
 * x[r * per + j] *= w[r] for r < rows, j < per (device arrays; w [rows]): each
 * sample's block of a batched gradient scaled by its weight, e.g. dL_b/dz by
 * the dObj/dL_b that gsparc_confidence writes (Eq. 5).
 */
int gsparc_scale_rows(int32_t rows, int64_t per, const float* w, float* x, void* stream);

/*
 * Polls a pipeline wait of the tensor-core compositing kernels
 * (gsparc_render_fwd_tc, gsparc_render_fwd_l2_tc, gsparc_render_csi_tc,
 * gsparc_render_bwd_tc, gsparc_render_bwd_tc_balanced) makes before it gives up
 * and the call reports GSPARC_ERR_TIMEOUT; 0 restores the default (2^22 polls,
 * well above any wait of a healthy launch).  Process-wide; read when a call
 * enqueues its kernel.  Returns the previous setting.  Meant for tests of the
 * timeout path: a small bound makes a wait expire without a fault or a hang.
 * Bounds below 1024 are counted in non-blocking polls (mbarrier.test_wait), so
 * that a bound of 1 ends every wait whose phase is not already complete; larger
 * bounds poll with the suspending mbarrier.try_wait.
 */
uint32_t gsparc_set_wait_limit(uint32_t polls);

/*
 * Launch overlap (programmatic dependent launch), process-wide.  `groups` is a
 * mask of the GSPARC_OVERLAP_* groups below (GSPARC_OVERLAP_ALL, the default,
 * or 0 for none).  The kernels of a group in the mask, which follow another
 * kernel of the library on a stream, are launched so that they may be
 * scheduled while the kernel before them is still running; each waits on the
 * device, before it touches any buffer, until that kernel has completed and
 * its writes are visible.  Results are the same either way (bit for bit where
 * the call is deterministic); outside the mask a launch is an ordinary one.
 * Read when a call enqueues its kernels, so it also holds inside a CUDA graph
 * captured while it was set.  Returns the previous mask.
 */
#define GSPARC_OVERLAP_BIN_SORT 1   /* gsparc_bin_sort: tile emit and sort      */
#define GSPARC_OVERLAP_FORWARD 2    /* the compositing forward kernels          */
#define GSPARC_OVERLAP_SCHEDULE 4   /* the balanced backward's schedule        */
#define GSPARC_OVERLAP_BACKWARD 8   /* the compositing backward walks          */
#define GSPARC_OVERLAP_NETWORK 16   /* gsparc_attr_mlp_bwd (FP32, tensor-core)  */
#define GSPARC_OVERLAP_ALL 31
int32_t gsparc_set_launch_overlap(int32_t groups);

/*
 * Synchronise `stream`, then return the value of the device status word
 * (GSPARC_OK if no device-side condition was raised) or GSPARC_ERR_CUDA if
 * the stream reports an error.  d_status may be NULL (stream check only).
 */
int gsparc_check(const int32_t* d_status, void* stream);

/* Human-readable text of a status code (static storage). */
const char* gsparc_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* GSPARC_H */
