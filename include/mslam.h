/*
 * mslam.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of MASt3R-SLAM (Murai, Dexheimer, Davison, arXiv 2412.12392):
 * iterative projective matching of two-view pointmaps (Sec. 3.2) feeding a
 * ray-error Sim(3) Gauss-Newton over a keyframe graph (Sec. 3.3, Sec. 3.5).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Memory: every array argument is a DEVICE pointer owned by the caller
 *   unless its comment says "host".  The library allocates no device memory;
 *   scratch space comes from the caller's `workspace` (size from
 *   mslam_workspace_bytes).  Host memory is used only inside mslam_plan_*.
 * - Streams: `stream` is a cudaStream_t cast to void* (NULL = legacy default
 *   stream).  Compute calls only enqueue work; they never synchronise, so a
 *   sequence of them can be captured into a CUDA graph.
 * - Errors: argument errors are detected on the host and returned at once
 *   (nothing is enqueued); a failed launch returns MSLAM_ERR_CUDA.  Errors
 *   that only the GPU can see (a non-positive Cholesky pivot, a non-finite
 *   step) are written to the caller's per-graph `dev_status` array, read
 *   after synchronising.  mslam_last_error() describes the last host-side
 *   error of the calling thread.
 * - Pools: per-keyframe tensors (canonical pointmaps) are concatenated in
 *   keyframe order, H_k W_k pixels each ("keyframe pool"); per-edge tensors
 *   (the pair prediction's pointmaps, descriptors and confidences, and the
 *   matches) are concatenated in edge order, H_j W_j pixels per edge ("edge
 *   pool").  Pixels are row-major (n = v W + u).
 * - Pointmaps are [pixels, 3] (x, y, z) of the storage dtype; descriptors
 *   chunk-planar [d / c, pixels, c] (see mslam_match); confidences [pixels].  MSLAM_F32 stores float, MSLAM_F16
 *   stores IEEE half; all arithmetic is float (FP32) except the pose algebra,
 *   the per-edge block assembly and the Cholesky solve, which are FP64.
 * - Poses T_wc are [N, 8] FP64: translation (3), unit quaternion x y z w (4),
 *   scale (1), mapping a camera point X to s R X + t (Sec. 3.1, Eq. 1).
 *   Tangent vectors tau are [N, 7]: (rho, phi, sigma) with
 *   Exp(tau) = expm([[ [phi]x + sigma I, rho ], [0, 0]]) and the left-plus
 *   update T <- Exp(tau) o T (Eq. 1).
 */
#ifndef MSLAM_H
#define MSLAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSLAM_OK = 0,
  MSLAM_ERR_ARG = 1,       /* invalid argument (host check) */
  MSLAM_ERR_CUDA = 2,      /* CUDA launch or runtime error */
  MSLAM_ERR_NOT_PD = 3,    /* reduced system not positive definite (dev_status) */
  MSLAM_ERR_TIMEOUT = 4,   /* a bounded device wait gave up (dev_status) */
  MSLAM_ERR_NONFINITE = 5, /* non-finite step (dev_status) */
  MSLAM_ERR_RANGE = 6      /* size beyond a stated limit */
} mslam_status;

typedef enum { MSLAM_F32 = 0, MSLAM_F16 = 1 } mslam_dtype;

/* Launch forms: the plain form issues one launch per edge from a host loop;
 * the default (batched) form covers every edge of every graph in one
 * persistent launch per stage. */
#define MSLAM_FLAG_PER_EDGE 1u

/* Workspace kinds for mslam_workspace_bytes */
#define MSLAM_OP_LINEARIZE 1
#define MSLAM_OP_SOLVE 2
#define MSLAM_OP_BACKWARD 3
#define MSLAM_OP_PACK_F32 4 /* packed-match buffer of mslam_gn_pack, FP32 storage */
#define MSLAM_OP_PACK_F16 5 /* packed-match buffer of mslam_gn_pack, FP16 storage */
#define MSLAM_OP_STATS 6    /* reference-pixel bitmap of mslam_match_stats */
#define MSLAM_OP_TRACK 7    /* tile partials and per-edge counters of mslam_gn_track */
#define MSLAM_OP_MATCH 8    /* reference ray image of mslam_match (16 bytes per edge-pool pixel) */

/* Constants of the method.  The paper names these quantities without values
 * where marked "reading"; defaults are set by mslam_default_params. */
typedef struct {
  float sigma_ray;       /* sigma_r of the weight w(q, sigma^2) = sigma^2 / q (Sec. 3.3); reading 0.01 */
  float sigma_dist;      /* sigma of the "small weight" distance term (Sec. 3.3, 3.5); reading 0.1 */
  float huber_delta;     /* Huber threshold of the robust norm on whitened residuals; reading 1.345 */
  float q_min;           /* matches with q <= q_min get w = infinity, i.e. are dropped (Sec. 3.3); reading 1.5 */
  float lm_lambda;       /* Levenberg-Marquardt damping of the matching step (Sec. 3.2); reading 1e-8 */
  int32_t lm_iters;      /* matching iterations; Sec. 3.2: 10 suffice for almost all valid pixels */
  int32_t win_radius;    /* refinement window radius r: (2r+1)^2 candidates per level; reading 3 */
  int32_t n_levels;      /* coarse-to-fine refinement levels (0..4); reading 2 */
  int32_t win_dilation[4]; /* candidate spacing per level, coarse first; reading {2, 1} */
  float max_rel_dist3d;  /* match invalid if |X_ref[m] - x| > this * |x| (Sec. 3.2 "large distances in 3D"); reading 0.1 */
  double conv_tol;       /* a graph stops updating once max|tau| < conv_tol (Sec. 3.5 "terminates upon convergence") */
  /* Residual family of the Gauss-Newton cost (MSLAM_RES_*):
   *   RAY   ray + distance errors, Eq. backend_ray / Eq. track_ray (default);
   *   POINT 3D point error r = T_ij X_j,n - X_i,m, Eq. track_point, Supp. S1.1;
   *   PIXEL known pinhole calibration, Sec. 3.6: pixel error Pi(T_ij X_j,n) - p_m
   *         (Eq. backend_pixel, Supp. S1.3) plus the depth error
   *         (T_ij X_j,n)_z - (X_i,m)_z; p_m = (m mod W, m div W) of the reference
   *         image; a match counts only if (T_ij X_j,n)_z > 1e-3 |T_ij X_j,n|. */
  int32_t residual;
  float sigma_point;     /* sigma_p of the point error; reading 0.05 */
  float sigma_pixel;     /* sigma_Pi of the pixel error, pixels; reading 1.0 */
  float sigma_depth;     /* sigma of the small-weight depth term of PIXEL; reading 0.1 */
  float fx, fy, cx, cy;  /* pinhole calibration K of PIXEL (pixels; centre of pixel (u, v) at (u, v)) */
} mslam_params;

#define MSLAM_RES_RAY 0
#define MSLAM_RES_POINT 1
#define MSLAM_RES_PIXEL 2

/* Fill `p` with the default readings listed above. */
void mslam_default_params(mslam_params* p);

/* Human-readable description of the calling thread's last host-side error. */
const char* mslam_last_error(void);

/* Library version string. */
const char* mslam_version(void);

/* ------------------------------------------------------------------------ */
/* Graph plan: the static structure of one or more keyframe graphs.         */
/* ------------------------------------------------------------------------ */
/* A plan holds the keyframe sizes, the directed edge list (Sec. 3.4: edges
 * are added in both directions), the pools' offsets, the work tiles of the
 * batched kernels and the symbolic block-sparse Cholesky factorisation of
 * each graph's 7N system with its first keyframe fixed (Sec. 3.5), ordered
 * by minimum degree.  It is built on the host once per edge structure.
 *
 *   N            number of keyframes (poses), >= 1
 *   kf_hw        host [N, 2] int32: H, W of each keyframe (2 <= H, W <= 8192)
 *   E            number of directed edges, >= 0
 *   edges        host [E, 2] int32: (i, j) = (reference keyframe, query
 *                keyframe); i != j, same graph, same image size
 *   graph_of_kf  host [N] int32 graph id in [0, G) or NULL (one graph).  The
 *                lowest-indexed keyframe of each graph is its fixed pose.
 *   out          receives the plan; destroy with mslam_plan_destroy.
 * Errors: MSLAM_ERR_ARG on any inconsistency, MSLAM_ERR_RANGE if host memory
 * for the plan's tables cannot be allocated (nothing is created either way). */
typedef struct mslam_plan mslam_plan;
mslam_status mslam_plan_create(int32_t N, const int32_t* kf_hw, int32_t E, const int32_t* edges,
                               const int32_t* graph_of_kf, mslam_plan** out);
void mslam_plan_destroy(mslam_plan* plan);

/* Launch-shape options of a plan (no effect on results beyond FP32
 * summation order), chosen by the caller or an autotuner:
 *   lin_tile           pixels per linearisation work tile: a multiple of 256
 *                      in [1024, 65536] (default 8192)
 *   lin_blocks_per_sm  resident blocks per SM of the persistent
 *                      linearisation launches, 1..32, or 0 for the
 *                      occupancy maximum (default 0)
 *   match_block_w      width of a 256-thread match block: 4, 8, 16, 32, 64,
 *                      128 or 256 (default 32, i.e. 32 x 8 threads)
 *   lin_form, solve_form  kernel forms, described at the fields
 * mslam_plan_create uses the defaults; mslam_plan_create_ex takes options
 * (NULL = defaults).  Errors: MSLAM_ERR_ARG for an option out of range, and
 * those of mslam_plan_create. */
typedef struct {
  int32_t lin_tile;
  int32_t lin_blocks_per_sm;
  int32_t match_block_w;
  int32_t lin_form;  /* packed linearisation of the FP16 ray family: 0 = records streamed through
                        shared memory by bulk asynchronous copies, one pipeline per block, and
                        evaluated two at a time with paired FP32 instructions, 1 = per-thread
                        register pipeline, 2 = the streamed form with one pipeline per warp (a warp
                        takes whole tiles; suits tiles of 1024-4096 pixels), 3 = the register
                        pipeline with each thread's next batch of records prefetched by asynchronous
                        copies into a 16 KB shared-memory buffer per block (the same sums in the same
                        order as form 1; default).  FP32 storage and the other residual families
                        always use the register pipeline. */
  int32_t solve_form;  /* 0 = FP32 factorisation of the diagonally scaled system with FP64 iterative
                          refinement to the FP64 solution (default; graphs it declines go to the FP64
                          factorisation), 1 = FP64 factorisation only */
  int32_t match_form;  /* refinement windows of mslam_match: 0 = each query thread scores its own window
                          on the FP32 pipe, reading the candidates from global memory (default), 1 = the
                          queries of a warp that share window rows are grouped and their windows scored
                          together on the tensor cores (same decisions up to the FP32 summation order of
                          the scores), 2 = per level, the block copies the box that holds its queries'
                          windows (at most 48 KB of descriptors) into shared memory with bulk
                          asynchronous copies and each query scores its window from there (from global
                          memory when its window falls outside the box): results bit-identical to form
                          0.  Forms 1 and 2 need FP16 storage and win_radius 3; other cases use form 0. */
  int32_t match_ppt;   /* query pixels per thread of mslam_match, 1 or 2 (default 1): a block of
                          match_block_w x (256 / match_block_w) threads covers match_ppt times as many
                          rows, each thread taking its queries 256 / match_block_w rows apart */
  int32_t wait_limit;  /* polls of every bounded device wait on an asynchronous copy (the streamed
                          linearisation forms, the staged match form) before it gives up: 0 = the
                          default 2^24 (about a second), > 0 = that many; < 0 = give up at once without
                          issuing any copy (so that nothing is in flight), which exercises the timeout
                          path in tests.  A staged match block whose wait gives up reads that level's
                          windows from global memory and stages nothing more: the result is unchanged */
} mslam_plan_opts;
void mslam_default_plan_opts(mslam_plan_opts* opts);
mslam_status mslam_plan_create_ex(int32_t N, const int32_t* kf_hw, int32_t E, const int32_t* edges,
                                  const int32_t* graph_of_kf, const mslam_plan_opts* opts, mslam_plan** out);

/* Bytes of device memory the plan's tables need, and their upload into a
 * caller-owned device buffer `dev` (>= 256-byte aligned) on `stream`.  The
 * buffer must outlive every call that uses the plan.  The host staging copy
 * is complete when the call returns. */
size_t mslam_plan_device_bytes(const mslam_plan* plan);
mslam_status mslam_plan_upload(mslam_plan* plan, void* dev, size_t bytes, void* stream);

/* Pool sizes: sum of H_k W_k over keyframes; sum of H_j W_j over edges. */
int64_t mslam_plan_kf_pixels(const mslam_plan* plan);
int64_t mslam_plan_edge_pixels(const mslam_plan* plan);
int32_t mslam_plan_num_graphs(const mslam_plan* plan);
/* Host copies of the structure: kf_off [N + 1] and e_off [E + 1] pixel
 * offsets of the pools; order [N] = elimination position of each keyframe
 * within its graph (-1 for the fixed keyframe); counts [4] = non-zero 7x7
 * blocks of L, update triples, work tiles of the linearisation, match blocks. */
void mslam_plan_offsets(const mslam_plan* plan, int64_t* kf_off, int64_t* e_off);
void mslam_plan_stats(const mslam_plan* plan, int32_t* order, int64_t* counts);

/* Scratch bytes a call of kind `op` (MSLAM_OP_*) needs for this plan. */
size_t mslam_workspace_bytes(const mslam_plan* plan, int32_t op);

/* ------------------------------------------------------------------------ */
/* (a1) The ray image, Sec. 3.1 (generic central camera).                     */
/* ------------------------------------------------------------------------ */
/* R[p] = psi(X[p]) = X[p] / |X[p]| for n_pix points X [n_pix, 3] of dtype dt
 * (FP32 or FP16), written to R [n_pix, 3] of the same dtype (device memory,
 * R may equal X); a zero or non-finite point gives the zero ray.  The norm
 * is formed in FP32 with the hardware reciprocal square root, exactly as
 * mslam_match evaluates the rays at its bilinear taps (it does not need this
 * image: it normalises the four taps of each iteration on the fly).
 * Errors: MSLAM_ERR_ARG (NULL pointer, negative size), MSLAM_ERR_CUDA. */
mslam_status mslam_ray_image(mslam_dtype dt, int64_t n_pix, const void* X, void* R, void* stream);

/* ------------------------------------------------------------------------ */
/* (a1-a3) Projective matching with feature refinement, Sec. 3.2, Eq. 2.     */
/* ------------------------------------------------------------------------ */
/* For every query pixel n of every edge e = (i, j) in [edge_begin, edge_end)
 * (-1, -1 = all edges):
 *   a1  the reference camera model psi(X_ref) = X_ref / |X_ref| (Sec. 3.1),
 *       evaluated at the four bilinear taps each iteration (a zero or
 *       non-finite reference point has the zero ray);
 *   a2  x = X_qry[n]; p starts at init_idx[n] (if init_idx != NULL and
 *       init_idx[n] >= 0) else at n itself (the identity map, Sec. 3.2), and
 *       takes lm_iters steps (J^T J + lm_lambda I) dp = -J^T r of the ray
 *       error r = R(p) - psi(x), R bilinear in the stored rays of the cell
 *       (clamp(floor u, 0, W-2), clamp(floor v, 0, H-2)), p clamped to the
 *       image after each step;
 *   a3  p is rounded half-up to a pixel, refined over n_levels windows of
 *       (2 win_radius + 1)^2 candidates spaced win_dilation[l] apart to the
 *       maximum descriptor dot product <D_qry[n], D_ref[c]> (first maximum in
 *       row-major order), and invalidated if x is zero/non-finite or
 *       |X_ref[m] - x| > max_rel_dist3d |x|; q = sqrt(Q_ref[m] Q_qry[n]).
 * Arguments (edge pools, dtype dt): X_ref, X_qry [P, 3]; D_ref, D_qry in the
 * chunk-planar layout [d / c, P, c] with c = 16 bytes of elements (8 halves
 * or 4 floats): channel k of pool pixel p is element ((k / c) P + p) c + k % c
 * (so a warp reading one chunk of neighbouring pixels reads contiguous
 * memory); d in {16, 24, 32}, 16-byte aligned; Q_ref, Q_qry [P]; init_idx [P]
 * int32 or NULL; outputs idx_out [P] int32 (m within the reference image,
 * -1 = invalid) and q_out [P] (dt; 0 where invalid).
 * n_valid, n_unique: [E] int32 or both NULL: the keyframe-criterion counts
 * of Sec. 3.4 (those of mslam_match_stats) taken in the matching epilogue
 * for the edges matched (other entries untouched); they need the workspace.
 * workspace: NULL, or >= mslam_workspace_bytes(plan, MSLAM_OP_MATCH) bytes,
 * 256-byte aligned: the call then first writes the unit rays psi(X_ref) of
 * the edges' reference pixels there (a1 as an image of float4, FP32, the same
 * arithmetic as at the taps) and the LM taps read them instead of
 * normalising four points per iteration; the result is identical.
 * flags: MSLAM_FLAG_PER_EDGE = one launch per edge, else one launch.
 * Errors: MSLAM_ERR_ARG for a null or misaligned pointer, unsupported d,
 * bad parameters or a workspace that is too small; MSLAM_ERR_CUDA if a
 * launch fails. */
mslam_status mslam_match(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, int32_t d,
                         const void* X_ref, const void* X_qry, const void* D_ref, const void* D_qry,
                         const void* Q_ref, const void* Q_qry, const int32_t* init_idx, int32_t* idx_out,
                         void* q_out, int32_t* n_valid, int32_t* n_unique, int32_t edge_begin, int32_t edge_end,
                         void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/* Descriptor layout for mslam_match: D [n_pix, d] row-major (the natural
 * layout a network writes) -> the chunk-planar layout, c = 16 bytes of
 * elements (8 halves or 4 floats): chunk k of source pixel p goes to element
 * ((k * dst_pix_stride + p) * c) of dst, so dst_pix_stride = n_pix gives
 * [d / c, n_pix, c], and dst_pix_stride = P with dst pointing at pixel p0 of
 * a [d / c, P, c] pool fills pixels [p0, p0 + n_pix) of it.  A copy, no
 * arithmetic.  src and dst are device buffers of dtype dt (16-byte aligned,
 * not overlapping), d in {16, 24, 32}, dst_pix_stride >= n_pix.
 * Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA. */
mslam_status mslam_desc_to_chunked(mslam_dtype dt, int32_t d, int64_t n_pix, const void* src, void* dst,
                                   int64_t dst_pix_stride, void* stream);

/* Keyframe criterion of Sec. 3.4 (next stage after matching): per edge, the
 * number of valid matches (idx >= 0) and the number of distinct reference
 * (keyframe) pixels they hit; tracking adds a keyframe when either, as a
 * fraction of the image, falls below omega_k (0.333 in the paper's setup).
 * idx: edge pool [P] int32 from mslam_match; outputs n_valid [E] and
 * n_unique [E] int32 (exact integer counts).  workspace >=
 * mslam_workspace_bytes(plan, MSLAM_OP_STATS), 256-byte aligned (a bitmap,
 * cleared by the call).  Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA. */
mslam_status mslam_match_stats(const mslam_plan* plan, const int32_t* idx, int32_t* n_valid, int32_t* n_unique,
                               void* workspace, size_t ws_bytes, void* stream);

/* The keyframe criterion of Sec. 3.4 on those counts (host function, no
 * GPU work: the decision steers the caller's host-side control flow): edge e
 * needs a new keyframe when n_valid[e] / n_query[e] < omega_k or
 * n_unique[e] / n_query[e] < omega_k (both in FP64; an edge with no query
 * pixels always needs one).  omega_k is 0.333 in the paper's evaluation
 * setup (Supp. S4).  All arrays are HOST memory of E entries; needed[e] is
 * set to 1 or 0.  Errors: MSLAM_ERR_ARG (NULL array with E > 0, E < 0, or
 * omega_k not in [0, 1]). */
mslam_status mslam_keyframe_criterion(int32_t E, const int32_t* n_valid, const int32_t* n_unique,
                                      const int64_t* n_query, double omega_k, int32_t* needed);

/* ------------------------------------------------------------------------ */
/* (a4-a5) Linearisation of the ray-error cost, Eq. backend_ray, Supp. S1.   */
/* ------------------------------------------------------------------------ */
/* For every edge e = (i, j) and every query pixel n with idx[n] = m >= 0 and
 * q[n] > q_min: x = T_ij X_canon_j[n] with T_ij = T_i^-1 T_j, y =
 * X_canon_i[m]; residuals r = psi(x) - psi(y) (3) and r_d = |x| - |y| (Supp.
 * S1.2); weights lambda = q / sigma^2 per term with one Huber IRLS weight on
 * the whitened ray residual norm and one on the distance residual; relative
 * Jacobians [(I - u u^T)/|x|, -[x]x/|x|, 0] and [u^T, 0, |x|] (u = x/|x|)
 * reduced per edge in FP32 (per-thread then tree sums, FP64 across tiles),
 * then mapped to the 14 x 14 block with Ad_{T_i^-1} (Supp. S1.4): H_ii = H_jj =
 * Ad^T H_rel Ad, H_ij = H_ji = -Ad^T H_rel Ad, g_i = -Ad^T g_rel,
 * g_j = Ad^T g_rel.
 * Arguments: T_wc [N, 8] FP64; X_canon keyframe pool [Pk, 3] (dt); idx, q
 * edge pools [P] (int32, dt).  Outputs: H_blocks [E, 14, 14] FP32 row-major
 * (rows/cols 0..6 = pose i, 7..13 = pose j), g_blocks [E, 14] FP32, cost [E]
 * FP64 (sum of Huber costs), n_valid [E] int32 or NULL (matches used).
 * workspace >= mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE), 256-byte
 * aligned.  flags: MSLAM_FLAG_PER_EDGE = plain form (a host loop of
 * per-edge launches), else one persistent launch over all tiles.
 * Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA. */
mslam_status mslam_gn_linearize(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, const double* T_wc,
                                const void* X_canon, const int32_t* idx, const void* q, float* H_blocks,
                                float* g_blocks, double* cost, int32_t* n_valid, void* workspace,
                                size_t ws_bytes, uint32_t flags, void* stream);

/* Packed form of the same linearisation.  The matches and the canonical
 * pointmaps do not change during the Gauss-Newton iterations of Sec. 3.5,
 * so mslam_gn_pack gathers, once, the inputs of every match used by
 * Eq. backend_ray (idx[n] >= 0 and q[n] > q_min): per work tile of the plan,
 * in pixel order, one record {X_j[n], X_i[m], q[n]} of the storage dtype
 * (16 bytes in FP16, 32 in FP32) plus a per-tile count.  The values are
 * copied bit for bit, so mslam_gn_linearize_packed computes exactly the sums
 * of mslam_gn_linearize (up to FP32 summation order) while streaming the
 * records with coalesced loads.  packed: caller device buffer of at least
 * mslam_workspace_bytes(plan, MSLAM_OP_PACK_F16 or _F32) bytes, 256-byte
 * aligned; it must be re-packed whenever X_canon, idx or q change.  The
 * record layout depends on the residual family (the pixel family stores
 * (u_m, v_m, depth of X_i[m]) in place of X_i[m]), so both calls take the
 * same parameters.  Other arguments and outputs as mslam_gn_linearize, plus
 * dev_status [G] int32 (the array mslam_gn_solve takes) or NULL: the
 * streamed forms (plan option lin_form 0 and 2) wait for their asynchronous
 * record copies with bounded waits (plan option wait_limit); if one gives
 * up, the launch's blocks are written as NaN, every graph of the launch gets
 * MSLAM_ERR_TIMEOUT in dev_status (which mslam_gn_solve then skips, leaving
 * its poses unchanged) and the kernel returns after its copies in flight
 * have landed.  Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA. */
mslam_status mslam_gn_pack(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, const void* X_canon,
                           const int32_t* idx, const void* q, void* packed, size_t packed_bytes, void* stream);
mslam_status mslam_gn_linearize_packed(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                       const double* T_wc, const void* packed, size_t packed_bytes, float* H_blocks,
                                       float* g_blocks, double* cost, int32_t* n_valid, int32_t* dev_status,
                                       void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/* mslam_gn_linearize without a workspace argument.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory --
 * e.g. a tracking loop with a fixed per-frame time budget, where cudaMalloc
 * may synchronise the device and stall the frame, or host code whose device
 * memory is owned by another allocator that hands out no raw scratch
 * buffers.  It uses a scratch array built into the library (4 MiB, held on
 * every GPU that loads the library until the process exits) and allocates
 * nothing; inputs and outputs are the caller's, exactly as in
 * mslam_gn_linearize.  The first call in a device's context looks up that
 * context's address of the array (cudaGetSymbolAddress, with the device
 * current; looked up again if the device's context has changed, e.g. after
 * cudaDeviceReset) and so should come before any stream capture on that
 * device.  All calls on a device share the array and every call rewrites
 * what it reads, so nothing needs clearing; calls whose GPU work overlaps
 * (e.g. on two streams) race on it and must be serialised.
 * Errors: MSLAM_ERR_RANGE if the plan needs more scratch than the array
 * holds (26,214 work tiles of 40 floats: about 26,000 tiles, i.e. 215 M
 * query pixels with the default 8,192-pixel tiles), otherwise as
 * mslam_gn_linearize. */
mslam_status mslam_gn_linearize_noalloc(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                        const double* T_wc, const void* X_canon, const int32_t* idx, const void* q,
                                        float* H_blocks, float* g_blocks, double* cost, int32_t* n_valid,
                                        uint32_t flags, void* stream);

/* ------------------------------------------------------------------------ */
/* (a6-a8) Gauss-Newton solve with the first pose fixed, Sec. 3.5.           */
/* ------------------------------------------------------------------------ */
/* Per graph: assemble the 14 x 14 edge blocks into the block-sparse 7N
 * system in FP64 (each block summed in edge order), drop the graph's first
 * keyframe (gauge), factor with a block Cholesky in the plan's
 * minimum-degree order, solve (J^T W J) tau = -J^T W r (Eq. gauss_newton)
 * and retract every other pose, T_k <- Exp(tau_k) o T_k, in FP64.
 * Arguments: H_blocks, g_blocks from mslam_gn_linearize; T_wc [N, 8] FP64
 * updated in place (the fixed poses are never written); tau [N, 7] FP64
 * output or NULL; dev_status [G] int32, zeroed by the caller before the
 * first iteration: a graph whose entry is non-zero is skipped.  The solve
 * writes 1 once max|tau| < conv_tol (converged), MSLAM_ERR_NOT_PD if a pivot
 * is not above 1e-12 times its assembled diagonal entry (the pose update is
 * then skipped), MSLAM_ERR_NONFINITE if the step is not finite.
 * workspace >= mslam_workspace_bytes(plan, MSLAM_OP_SOLVE).
 * Errors (returned): MSLAM_ERR_ARG, MSLAM_ERR_CUDA. */
mslam_status mslam_gn_solve(const mslam_params* p, const mslam_plan* plan, const float* H_blocks,
                            const float* g_blocks, double* T_wc, double* tau, int32_t* dev_status, void* workspace,
                            size_t ws_bytes, void* stream);

/* Kernel launches one mslam_gn_solve call enqueues on this plan: 3 with the
 * mixed-precision solve (plan option solve_form 0: FP32 factorisation of the
 * diagonally scaled system, FP64 iterative refinement; the FP32 factor sits
 * in shared memory, or, when the largest graph's factor does not fit there,
 * every graph's factor is worked on in place in the workspace): its
 * assembly-and-scaling kernel, the solve, and an FP64 kernel for any graph
 * it declines; 1 (FP64 only) with solve_form 1 or when not even the solve's
 * vectors and tables fit in shared memory. */
int32_t mslam_gn_solve_launches(const mslam_plan* plan);

/* ------------------------------------------------------------------------ */
/* (a9) Adjoint of the weighted cost (project form; not in the paper).      */
/* ------------------------------------------------------------------------ */
/* Gradient of L = dL_dcost * E_g(T, X_canon, q) + dL_dtau . tau(T, X_canon, q)
 * with respect to the canonical pointmaps and the match confidences, where
 * E_g is Eq. backend_ray at the poses T_wc (matches and the q_min mask held
 * fixed, Huber weights differentiated) and tau = -H^-1 g is one
 * Gauss-Newton step from T_wc (Eq. gauss_newton).  The per-pixel residuals
 * and Jacobians are recomputed, not stored.  The step term's two solves
 * (tau and b = H^-1 dL_dtau) follow the plan's solve_form: the FP32 factor
 * of the Jacobi-scaled system refined with FP64 residuals (kept in the
 * workspace between the two), the FP64 factorisation for the graphs that
 * path declines and with solve_form 1.
 * Arguments: as mslam_gn_linearize, plus H_blocks and g_blocks of the
 * linearisation at T_wc (needed when dL_dtau != NULL), dL_dtau [N, 7] FP64
 * device or NULL, dL_dcost host scalar; outputs dL_dX [Pk, 3] FP32 and dL_dq
 * [P] FP32, overwritten.  workspace >= mslam_workspace_bytes(plan,
 * MSLAM_OP_BACKWARD).  Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA; a singular
 * system sets dev_status[g] = MSLAM_ERR_NOT_PD. */
mslam_status mslam_gn_backward(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, const double* T_wc,
                               const void* X_canon, const int32_t* idx, const void* q, const float* H_blocks,
                               const float* g_blocks, const double* dL_dtau, double dL_dcost, float* dL_dX,
                               float* dL_dq, int32_t* dev_status, void* workspace, size_t ws_bytes,
                               void* stream);

/* Adjoint of one whole Gauss-Newton step T' = Exp(tau) o T with tau =
 * -H(T)^-1 g(T) (Eq. gauss_newton, Eq. 1; project form, not in the paper),
 * so that unrolled steps can be chained: the gradient of
 *   L = dL_dcost * E_g(T) + dL_dtau . tau + <dL_dTnew, T'>
 * with respect to X_canon, q and the poses T_wc.  Poses enter through every
 * match's x = T_i^-1 T_j X_j[n], through the adjoint Ad_{T_i^-1} that maps
 * each edge's relative system to its 14 x 14 block, and through the
 * retraction (left Jacobian of Exp); matches and the q_min mask are held
 * fixed, the Huber weights are differentiated.  Pose gradients are given
 * and returned in the [N, 8] embedding (t, q, s): G with J8^T G = dL/deta
 * for the left perturbation T -> Exp(eta) T (J8 = d(t, q, s)/d eta) and no
 * component along the quaternion's norm direction.
 * Arguments: as mslam_gn_backward, plus dL_dTnew [N, 8] FP64 (device, the
 * gradient on the updated poses) or NULL, and the output dL_dT [N, 8] FP64
 * (device, required).  H_blocks, g_blocks (the linearisation at T_wc) and
 * dev_status are required.  tau is recomputed from H and g (as in
 * mslam_gn_backward, to the FP64 solution).  The
 * gradient of the fixed (first) keyframe's pose is returned too: moving it
 * moves every other pose's step.  Errors: MSLAM_ERR_ARG, MSLAM_ERR_CUDA; a
 * singular system sets dev_status[g] = MSLAM_ERR_NOT_PD (the gradients of
 * that graph are then not defined). */
mslam_status mslam_gn_step_backward(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                    const double* T_wc, const void* X_canon, const int32_t* idx, const void* q,
                                    const float* H_blocks, const float* g_blocks, const double* dL_dTnew,
                                    const double* dL_dtau, double dL_dcost, float* dL_dX, float* dL_dq,
                                    double* dL_dT, int32_t* dev_status, void* workspace, size_t ws_bytes,
                                    void* stream);

/* ------------------------------------------------------------------------ */
/* Tracking, Sec. 3.3: the frame's Gauss-Newton loop in one launch per       */
/* iteration.                                                                 */
/* ------------------------------------------------------------------------ */
/* For plans in which every graph is one keyframe (its gauge) and one frame
 * joined by one edge (a tracking problem; several are solved side by side):
 * n_iters iterations of a4-a8 on the ray family, each one launch.  Every
 * block linearises one tile of packed records (mslam_gn_pack) against the
 * relative pose it forms from T_wc, stores the tile's sums, and the block
 * that completes an edge's last tile adds the edge's tile sums in tile order
 * in FP64, maps them to the frame's 7 x 7 system with the adjoint (the
 * gauge removed), solves it by FP64 Cholesky and retracts the frame's pose
 * in T_wc (Exp(tau) o T).  dev_status [G] as in mslam_gn_solve: a graph
 * with status > 0 is skipped; 1 is written once max|tau| < conv_tol,
 * MSLAM_ERR_NOT_PD for a pivot that is not positive.  The result equals
 * the linearise + solve loop up to the rounding of the 14 x 14 blocks,
 * which stay FP64 here.  workspace >= mslam_workspace_bytes(plan,
 * MSLAM_OP_TRACK), 256-byte aligned.  Errors: MSLAM_ERR_ARG (a plan that is
 * not of this form, a residual family other than the ray family, n_iters
 * < 0, NULL or misaligned pointers), MSLAM_ERR_CUDA. */
mslam_status mslam_gn_track(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, double* T_wc,
                            const void* packed, size_t packed_bytes, int32_t n_iters, int32_t* dev_status,
                            void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Pointmap fusion, Sec. 3.3 (next stage after tracking).                    */
/* ------------------------------------------------------------------------ */
/* Running weighted average of the keyframe's canonical pointmap:
 *   X~ <- (C~ X~ + C (T_kf X)) / (C~ + C),  C~ <- C~ + C,
 * per pixel, T_kf = T_wc[k]^-1 T_wc[f] computed on the device from the pose
 * array (no host round trip after the tracking solve).  X_canon_k [n_pix, 3]
 * and C_canon_k [n_pix] are keyframe k's canonical pointmap and confidence
 * (updated in place); X_kf [n_pix, 3] and C_kf [n_pix] the keyframe's points
 * as predicted with frame f, in frame f's coordinates, and their
 * confidences; all of dtype dt, pixel-aligned with the keyframe.  A pixel
 * whose prediction is non-finite, zero or has a confidence that is not
 * positive is left unchanged.  Errors: MSLAM_ERR_ARG (NULL pointer, k == f,
 * negative size), MSLAM_ERR_CUDA. */
mslam_status mslam_fuse(mslam_dtype dt, const double* T_wc, int32_t k, int32_t f, int64_t n_pix, void* X_canon_k,
                        void* C_canon_k, const void* X_kf, const void* C_kf, void* stream);

/* Known calibration, Sec. 3.6 (first of its two changes): before a
 * canonical pointmap is used, keep only the depth z of each point and place
 * the point on its pixel's ray of the pinhole camera,
 *   X[p] <- z ((u - cx) / fx, (v - cy) / fy, 1),  (u, v) = (p mod W, p div W).
 * X: [n_images, H, W, 3] of dt (FP32 or FP16), in place, device memory.
 * Pairs with residual = MSLAM_RES_PIXEL and the same fx, fy, cx, cy.
 * Errors: MSLAM_ERR_ARG (NULL pointer, negative size, fx or fy not positive
 * or a non-finite calibration), MSLAM_ERR_CUDA. */
mslam_status mslam_calib_backproject(mslam_dtype dt, int32_t n_images, int32_t H, int32_t W, float fx, float fy,
                                     float cx, float cy, void* X, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MSLAM_H */
