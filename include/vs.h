/*
 * vs.h -- C ABI of the GB300 (sm_103a) k-shell renderer ("Volumetric
 * Surfaces", arXiv 2409.02482).
 *
 * A baked Volumetric-Surfaces asset is k nested, semi-transparent,
 * UV-textured triangle meshes ("shells").  A frame rasterizes every shell in
 * a fixed outer-to-inner order, each with its own nearest-hit test (Fig. 3c:
 * only the first intersection with each surface is sampled), samples each
 * hit's texture bilinearly at texel centres (Fig. 5), decodes spherical
 * harmonics with the view direction (Sec. 3 "Texturing Meshes"), and
 * alpha-composites the hits front to back (Eq. 6, with the transmittance of
 * Eq. 1 taken over the *earlier* layers only).  No sorting is involved: the
 * shell order is the blend order (Sec. 3 "Support Surfaces as Shells").
 * The backward pass is the texel gradient used by the paper's post-bake
 * texture fitting (Sec. 3 "Texturing Meshes").
 *
 * Conventions shared by all entry points
 * ---------------------------------------
 * Memory.  Every pointer named "device" is CUDA device memory owned by the
 *   caller; the library never allocates device memory.  Its only scratch is
 *   the caller's `workspace` (size from vs_workspace_size).  A workspace must
 *   be zero-filled once before its first use; afterwards calls keep it valid.
 *   Calls that share a workspace must not overlap on the GPU.
 * Streams.  Work is enqueued asynchronously on `stream` (NULL = the legacy
 *   default stream); no call synchronizes except vs_read_stats.
 * Errors.  Every call returns a vs_status; nothing aborts or throws across the
 *   ABI.  Argument errors are detected on the host before anything is
 *   enqueued.  Errors found on the device (a bounded wait that ran out,
 *   a malformed input detected while running) are recorded in the workspace
 *   and returned by vs_read_stats.  vs_last_error() gives a message for the
 *   calling thread's last failure.
 * Layouts.  Row-major, C order.  Shell 0 is the OUTERMOST; the library never
 *   reorders shells.  Triangles are counter-clockwise seen from outside
 *   (front faces).  Texel (x, y) is centred at UV ((x+1/2)/W, (y+1/2)/H),
 *   row 0 at v = 0, clamp-to-edge addressing, no mipmaps.
 * Cameras.  OpenCV pinhole: x right, y down, z forward; pixel (x, y) is
 *   sampled once at its centre (x + 1/2, y + 1/2).
 * Exactness.  Which triangle a pixel sees in each shell is decided in
 *   integer arithmetic after a fixed FP32 vertex transform (1/256-pixel
 *   snapping, top-left fill rule, exact depth-key interpolation, ties to the
 *   lower triangle index), so hit IDs are reproducible bit for bit.  Colours
 *   and gradients are FP32 (no FP64 on the GPU).
 */
#ifndef VS_H_
#define VS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vs_status;
#define VS_OK 0
#define VS_ERR_INVALID_ARG (-1) /* bad pointer, size, format or range     */
#define VS_ERR_CUDA (-2)        /* a CUDA runtime call failed              */
#define VS_ERR_UNSUPPORTED (-3) /* valid but not implemented combination   */
#define VS_ERR_WORKSPACE (-4)   /* workspace NULL, too small or misaligned */
#define VS_ERR_OVERFLOW (-5)    /* a size exceeds a documented limit       */
#define VS_ERR_TIMEOUT (-6)     /* a bounded device wait ran out           */

/* cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st* vs_stream_t;

typedef struct vs_ctx vs_ctx;       /* opaque: device id and its properties */
typedef struct vs_object vs_object; /* opaque: k shells (non-owning views)  */

/* Texel formats.
 * VS_TEX_RGBA_F32: float32 (r, g, b, alpha), used as stored.
 * VS_TEX_SH_F16:   float16 [a, r0, g0, b0, r1, g1, b1, ...]: one alpha logit
 *   and the (d+1)^2 RGB spherical-harmonic coefficients of degree d <= 3,
 *   coefficient-major with channels interleaved (the paper's baked layout
 *   stores coefficient i of every channel in image i, Sec. 3 "Baking
 *   Textures").  alpha = sigmoid(a), rgb = sigmoid(sum_m sh_m Y_m(v)) with v
 *   the unit ray direction and Y_m the real orthonormal SH (l = 1 band
 *   proportional to (y, z, x)), index m = l^2 + l + m'.
 *   C = 1 + 3 (d+1)^2 values: 4, 13, 28, 49 for d = 0..3.
 */
#define VS_TEX_RGBA_F32 0
#define VS_TEX_SH_F16 1
/* VS_TEX_SH_U8: the paper's deployed (baked) texels (Sec. 3 "Mixed
 *   Resolutions", "Squeezing and Quantization", "Baking Textures"): SH
 *   coefficients of degree d <= 3 for all four channels -- opacity is view
 *   dependent too: (r, g, b, alpha) = sigmoid(sum_m sh_{m,c} Y_m(v)) -- one
 *   byte q each, decoded as value_min + (value_max - value_min) q / 255.
 *   Band l (coefficients l^2 .. l^2 + 2l) is its own image of
 *   (tex_w >> l s) x (tex_h >> l s) texels, s = band_shift (s = 1: the
 *   paper's mixed resolutions, 2048^2 base colour down to 256^2 for band 3;
 *   s = 0: one resolution).  A texel of band l holds its 2l + 1 coefficients
 *   as (r, g, b, alpha) byte quadruples in coefficient order, padded to 4,
 *   16, 32, 32 bytes for l = 0..3; the bands follow each other in one buffer
 *   (`texels`), each starting on a 256-byte boundary (vs_baked_layout).
 *   Forward only: vs_render_backward and the backward of vs_render_batch
 *   return VS_ERR_UNSUPPORTED for these shells (the paper fits continuous
 *   textures and quantises when baking). */
#define VS_TEX_SH_U8 2

/* One shell.  All pointers are device memory, kept alive by the caller until
 * vs_free_shells. */
typedef struct {
  const float* pos;      /* [num_verts, 3] object = world space          */
  int32_t num_verts;     /* 3 <= num_verts <= 2^30                       */
  const float* uv;       /* [num_verts, 2]                                */
  const int32_t* tris;   /* [num_tris, 3] vertex indices, CCW = front    */
  int32_t num_tris;      /* 1 <= num_tris <= 2^31 - 2                    */
  const void* texels;    /* [tex_h, tex_w, texel_pitch] of the format's type;
                            VS_TEX_SH_U8: the band buffer, 16-byte aligned */
  int32_t tex_w, tex_h;  /* 1 .. 65536 each (VS_TEX_SH_U8: band 0; both
                            divisible by 2^(d * band_shift))               */
  int32_t format;        /* VS_TEX_*                                      */
  int32_t sh_degree;     /* 0..3 for the SH formats, ignored for RGBA     */
  int32_t texel_pitch;   /* values per texel in memory, >= C (padding ok);
                            ignored for VS_TEX_SH_U8                        */
  int32_t band_shift;    /* VS_TEX_SH_U8: 0..3, ignored otherwise         */
  float value_min;       /* VS_TEX_SH_U8: decode range, value_min <      */
  float value_max;       /*   value_max, both finite; ignored otherwise   */
  int32_t grad_pitch;    /* FP32 values per texel of this shell's gradient
                            arrays (vs_render_backward, vs_render_batch):
                            0 = texel_pitch, else >= C; lets the gradient
                            drop the texels' alignment padding (e.g. 28 for
                            SH degree 2 stored at texel_pitch 32).  Ignored
                            for VS_TEX_SH_U8                              */
} vs_shell_desc;

/* Layout of a VS_TEX_SH_U8 buffer (pure host arithmetic): for bands
 * l = 0..sh_degree, the byte offset, width, height and bytes per texel of
 * band l (entries past sh_degree are set to 0), and the buffer's total size.
 * Any output pointer may be NULL.  Errors: VS_ERR_INVALID_ARG for sizes out
 * of range or not divisible by 2^(sh_degree * band_shift). */
vs_status vs_baked_layout(int32_t tex_w, int32_t tex_h, int32_t sh_degree, int32_t band_shift,
                          int64_t band_offset[4], int32_t band_w[4], int32_t band_h[4],
                          int32_t band_stride[4], int64_t* total_bytes);

typedef struct {
  float world_to_cam[12]; /* row-major 3x4 [R | t]                        */
  float fx, fy, cx, cy;   /* pinhole intrinsics in pixels                  */
  float znear;            /* > 0: near plane in camera space; faces crossing
                             it are clipped there (z = znear), faces wholly
                             nearer are culled                            */
  int32_t width, height;  /* 1 .. 8192 each                                */
} vs_camera;

/* Flags (bitwise OR). */
#define VS_FLAG_LOSS_L2 (1u << 0)
/* Backward only: `grad_rgb` holds the TARGET image [H, W, 3] instead of a
 * gradient; the kernel uses dL/dC = 2 (C - target) / (3 H W), i.e. the
 * gradient of the mean squared error over pixels and RGB channels, computing
 * C itself from the hits, and adds L to `loss` when that pointer is set. */
#define VS_FLAG_LOSS_L1 (1u << 2)
/* Backward only, like VS_FLAG_LOSS_L2 with the pixel-wise L1 colour loss the
 * textures are fitted with (Sec. 3 "Texturing Meshes"): L = mean over pixels
 * and RGB channels of |C - target|, dL/dC = sign(C - target) / (3 H W) with
 * sign(0) = 0.  Setting both loss flags is VS_ERR_INVALID_ARG. */
#define VS_FLAG_ALPHA_ATTEN (1u << 1)
/* Transparency attenuation (Sec. 3 "Transparency Attenuation"): every
 * fragment's opacity is multiplied by alpha_w = 2 sigmoid(10 |v . n|) - 1,
 * v the unit ray direction of the pixel and n the unit normal of the hit
 * triangle, (p1 - p0) x (p2 - p0) of its stored world positions.  Applies to
 * vs_render, vs_render_backward (pass the same flags as the forward) and
 * vs_render_batch; the backward treats alpha_w as a constant of the texels.
 * Off by default: the paper defines it for blending during training and does
 * not say whether the baked renderer keeps it. */
#define VS_FLAG_TEST_STALL (1u << 30)
/* Test hook for failure detection: the persistent batch kernel's first
 * shading unit waits for a counter that nothing increments, with a short
 * spin limit, so the call ends with VS_ERR_TIMEOUT recorded in the
 * workspace.  The wait is bounded; the context stays usable. */

/* Limits. */
#define VS_MAX_SHELLS 16
#define VS_MAX_IMAGE_SIDE 8192

/* --- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (queries its properties; makes
 * no allocation).  Errors: VS_ERR_INVALID_ARG (ctx NULL), VS_ERR_CUDA (no
 * such device). */
vs_status vs_create(vs_ctx** ctx, int device);
vs_status vs_destroy(vs_ctx* ctx);

/* Message of the calling thread's last failed call ("" if none).  Valid
 * until the thread's next call into the library. */
const char* vs_last_error(void);

/* --- assets ---------------------------------------------------------------- */

/* Wraps k shells (index 0 = outermost) into an object.  Copies the
 * descriptors (host memory only); the device arrays stay the caller's.  The
 * first render with the object reads its vertex positions once (a
 * synchronous device-to-host copy: make that call before any stream
 * capture) to bound each shell; calls whose cameras keep every shell in
 * front of the near plane run kernels without the clipping code, the others
 * run the generic kernels that clip.  Reload the object if its positions
 * change.
 * Errors: VS_ERR_INVALID_ARG for k outside [1, VS_MAX_SHELLS], NULL
 * pointers, sizes out of range, unknown format, texel_pitch < C, SH degree
 * outside [0, 3]; for VS_TEX_SH_U8 also band_shift outside [0, 3], band
 * sizes not dividing, a decode range that is not finite and increasing, or
 * a buffer not 16-byte aligned. */
vs_status vs_load_shells(vs_ctx* ctx, const vs_shell_desc* shells, int32_t k, vs_object** out);
vs_status vs_free_shells(vs_ctx* ctx, vs_object* obj);

/* --- scratch ------------------------------------------------------------------ */

/* Bytes of workspace needed to render (and differentiate) the n_items
 * (object, camera) pairs in ONE vs_render_batch call; for n_items = 1 it
 * also covers vs_render / vs_render_backward of that pair.  Dominant terms
 * per item: 8 * k * H * W (per-shell visibility words) + 16 * sum(V)
 * (snapped vertices).  Pure host arithmetic.  Errors: VS_ERR_INVALID_ARG. */
vs_status vs_workspace_size(vs_ctx* ctx, const vs_object* const* objs, const vs_camera* cams,
                            int32_t n_items, uint32_t flags, size_t* bytes);

/* --- forward ------------------------------------------------------------------ */

/* Renders one object from one camera.
 *   bg        host float[3], background colour (NULL = black)
 *   out_rgba  device float32 [H, W, 4] = (C + T bg, 1 - T), T the
 *             transmittance left after the last shell
 *   hits      device int32 [k, H, W] shell-local triangle index of each
 *             shell's nearest front-facing hit, -1 = miss; may be NULL.
 *             The only state vs_render_backward needs.
 *   workspace device, >= vs_workspace_size(obj, cam, 1), 256-byte aligned
 * Launches, in order: the item-table upload, clear + vertex setup, raster,
 * shade + composite. */
vs_status vs_render(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg,
                    float* out_rgba, int32_t* hits, void* workspace, size_t ws_bytes,
                    uint32_t flags, vs_stream_t stream);

/* --- backward ------------------------------------------------------------------- */

/* Accumulates dL/d(texel values) into grad_texels given dL/d(output rgb).
 *   hits         device int32 [k, H, W] as written by vs_render for the same
 *                object, camera and texels
 *   grad_rgb     device float32 [H, W, 3] (or the target image with
 *                VS_FLAG_LOSS_L2 / VS_FLAG_LOSS_L1)
 *   grad_texels  host array of k device pointers, each float32
 *                [tex_h, tex_w, grad_pitch] (grad_pitch = texel_pitch
 *                unless the shell sets it); ADDED to (zero them first);
 *                padding values receive nothing
 *   loss         device float32 scalar, L added (with a loss flag only; may
 *                be NULL)
 * Transmittance is recomputed from the hits, not stored.  Gradients use
 * float atomics: summation order, hence the last bits, vary run to run. */
vs_status vs_render_backward(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam,
                             const float* bg, const int32_t* hits, const float* grad_rgb,
                             float* const* grad_texels, float* loss, void* workspace,
                             size_t ws_bytes, uint32_t flags, vs_stream_t stream);

/* --- per-layer buffers --------------------------------------------------------- */

/* vs_render plus every shell's own render buffers before blending, as in the
 * paper's render-buffer figures (Figs. S1/S3): `layers` is device float32
 * [k, H, W, VS_LAYER_FLOATS], 16-byte aligned; record (shell i, pixel) =
 *   [0..2] unit geometric normal of the hit face, (p1 - p0) x (p2 - p0) of
 *          its stored world positions normalised
 *   [3..4] texture coordinates (u, v) at the pixel (perspective-correct)
 *   [5]    opacity alpha_i (after VS_FLAG_ALPHA_ATTEN, if set)
 *   [6]    blending weight T_i alpha_i (the layer's contribution)
 *   [7..9] colour (r, g, b)
 *   [10..11] 0
 * all zero where shell i has no fragment.  The weights sum to the output
 * alpha, and sum_i weight_i rgb_i + (1 - alpha) bg is the output colour.  A
 * debugging aid: it runs the generic kernels.  Errors: as vs_render. */
#define VS_LAYER_FLOATS 12
vs_status vs_render_layers(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg, float* out_rgba,
                           int32_t* hits, float* layers, void* workspace, size_t ws_bytes, uint32_t flags,
                           vs_stream_t stream);

/* --- batch ------------------------------------------------------------------------ */

typedef struct {
  const vs_object* obj;
  vs_camera cam;
  float* out_rgba;            /* device [H, W, 4]; required               */
  int32_t* hits;              /* device [k, H, W] or NULL                 */
  const float* grad_rgb;      /* device [H, W, 3] (do_backward only)      */
  float* const* grad_texels;  /* host array of k device pointers (bwd)    */
  float* loss;                /* device scalar or NULL (loss flags)       */
} vs_batch_item;

/* Renders n items -- any mix of objects, shell counts, triangle counts and
 * resolutions -- in ONE persistent kernel launch (after small launches that
 * copy the item table into the workspace).  The items run in an order of
 * the library's choosing, for cache locality: grouped by object, and within
 * an object a nearest-neighbour chain of camera centres from its first item
 * (up to 4096 items per object; larger groups keep the given order).
 * Outputs do not depend on the order, gradient sums only through the
 * rounding order of their FP32 atomics.  Work units are handed out in a
 * fixed, skewed global order (stage s: vertex setup of item s, raster of
 * item s-1, shading of item s-2); a unit waits, with a bounded spin, only
 * for units handed out before it, so the launch cannot deadlock.  With do_backward, each pixel's forward result is
 * differentiated in the same unit (fused forward + backward) using
 * grad_rgb -- with a loss flag, the target image.  Forward outputs are
 * bit-identical to vs_render of each item.  All enqueued work is
 * capturable in a CUDA graph (the item table travels in kernel parameters).
 * Workspace: vs_workspace_size of all n items runs them in one launch.  A
 * smaller workspace runs them as consecutive launches over runs of items,
 * each run the longest that fits (e.g. hundreds of 4K views whose per-shell
 * visibility words would not all fit); results are
 * the same, the runs do not overlap.  Every item is checked before anything
 * is enqueued.
 * Errors: as vs_render; VS_ERR_INVALID_ARG for n < 1; VS_ERR_WORKSPACE when
 * a single item does not fit. */
vs_status vs_render_batch(vs_ctx* ctx, const vs_batch_item* items, int32_t n, const float* bg,
                          int32_t do_backward, void* workspace, size_t ws_bytes, uint32_t flags,
                          vs_stream_t stream);

/* --- batch tuning ---------------------------------------------------------------- */

/* Launch shape of vs_render_batch.  The paper's renderer has no such knobs
 * (a GL pipeline bins and tiles in fixed function); these are the work-unit
 * ("tile") sizes of the persistent kernel and its grid. */
typedef struct {
  int32_t raster_tris;    /* triangles per raster work unit: a power of two in
                             [32, 2048]                                       */
  int32_t shade_pixels;   /* pixels per shading work unit: a power of two in
                             [32, 4096]                                       */
  int32_t blocks_per_sm;  /* persistent blocks per SM (blocks of 160
                             threads with do_backward, else 256); 0 = the
                             occupancy maximum, else 1 .. that maximum
                             (larger values are clamped to it at launch)      */
  int32_t reserved;       /* must be 0                                        */
} vs_tuning;

/* The default: 256 triangles, 256 pixels, occupancy maximum. */
#define VS_TUNING_DEFAULT_RASTER_TRIS 256
#define VS_TUNING_DEFAULT_SHADE_PIXELS 256

/* Sets / reads the tuning vs_render_batch uses for batches whose largest
 * shell count is k_max (1 .. VS_MAX_SHELLS; setting also takes 0 = every
 * k_max) and the given do_backward.  Until set, the default applies.  The tuning changes launch
 * shape only: forward outputs stay bit-identical to vs_render.  The
 * arguments are checked before the context (VS_ERR_INVALID_ARG), so a bad
 * tuning is refused even with a NULL context.  The context's table is
 * guarded by a mutex. */
vs_status vs_set_batch_tuning(vs_ctx* ctx, int32_t do_backward, int32_t k_max, const vs_tuning* t);
vs_status vs_get_batch_tuning(vs_ctx* ctx, int32_t do_backward, int32_t k_max, vs_tuning* t);

/* Host-only coordinate-descent search over the tuning space: starting from
 * `start`, it sweeps raster_tris over {64, 128, 256, 512, 1024},
 * shade_pixels over {64, 128, 256, 512, 1024} and blocks_per_sm over
 * 1 .. max_blocks_per_sm one coordinate at a time, moving to the cheapest
 * value, until a sweep changes nothing (at most 4 sweeps).  `cost` returns
 * the cost (e.g. milliseconds) of one configuration; each configuration is
 * evaluated at most once.  Returns the cheapest configuration seen in *best
 * and the number of cost calls in *evaluations (may be NULL).  A cost that
 * is negative or NaN ends the search with VS_ERR_INVALID_ARG.  Needs no GPU;
 * vs_autotune_batch runs it with a timed launch as the cost. */
typedef double (*vs_cost_fn)(const vs_tuning* t, void* user);
vs_status vs_tune_search(const vs_tuning* start, int32_t max_blocks_per_sm, vs_cost_fn cost, void* user,
                         vs_tuning* best, int32_t* evaluations);

/* Autotunes vs_render_batch for this batch: vs_tune_search from the current
 * tuning, the cost of a configuration being the shortest of `repeats`
 * (1 .. 16) CUDA-event-timed launches after one untimed one.  Stores the
 * winner for (do_backward, largest k of the batch) in the context, returns
 * it in *best (may be NULL) and synchronises the stream.  The launches are
 * real: outputs are overwritten and, with do_backward, texel gradients and
 * losses ACCUMULATE over all of them -- zero them before the next real step.
 * The workspace's device counters (vs_read_stats) include these launches.
 * Not capturable (it synchronises); tune first, then capture.
 * Errors: as vs_render_batch; VS_ERR_INVALID_ARG for repeats out of range;
 * a device error recorded by any launch ends the search with that status. */
vs_status vs_autotune_batch(vs_ctx* ctx, const vs_batch_item* items, int32_t n, const float* bg,
                            int32_t do_backward, void* workspace, size_t ws_bytes, uint32_t flags,
                            vs_stream_t stream, int32_t repeats, vs_tuning* best);

/* --- neural texture (Sec. 3 "Texturing Meshes") -------------------------------- */

/* A texture as a function: a 2D multiresolution hash encoding (the trainable
 * positional encoding of Mueller et al. 2022) followed by an MLP of two
 * hidden ReLU layers and a linear output (the supplement's neural texture
 * architecture), evaluated at the texel centres ((i + 1/2)/W, (j + 1/2)/H)
 * of the target resolution -- "grounded", so the texture the renderer
 * samples bilinearly IS the prediction.  Definitions:
 *   level l resolution N_l = floor(base_res * growth^l); p = x N_l; corners
 *   floor(p) + {0,1}^2 with bilinear weights; table row of corner c: dense
 *   c0 + c1 (N_l + 1) if (N_l + 1)^2 <= T, else (c0 XOR c1 * 2654435761)
 *   mod T (uint32 arithmetic); feature f_l = sum w table[l, row, :];
 *   y = W2 relu(W1 relu(W0 f + b0) + b1) + b2.
 * Parameters: one device float32 vector, blocks in this order:
 *   table [L, T, F], W0 [H, L F], b0 [H], W1 [H, H], b1 [H], W2 [C, H], b2 [C]
 * (row-major).  The paper uses separate networks for colour and opacity:
 * write them to different channel ranges of one texel array (ch0). */
typedef struct {
  int32_t levels;        /* L: 1 .. 16                                    */
  int32_t features;      /* F per level: 1 .. 8                           */
  int32_t log2_table;    /* T = 2^log2_table rows per level: 2 .. 24      */
  int32_t base_res;      /* N_min >= 1                                     */
  float growth;          /* b in [1, 4]; N_l <= 2^20                       */
  int32_t hidden;        /* H: 1 .. 512                                    */
  int32_t out_ch;        /* C: 1 .. 256                                    */
  int32_t tensor_cores;  /* 0: FP32 layers (FP32 FMAs on the FP32 pipes, the
                            default); 1: the layer products shaped like the
                            forward (the three layers, and the adjoint's
                            activation gradients) on the tensor cores
                            (tcgen05, inputs rounded to TF32 -- 10-bit
                            mantissa, to nearest -- FP32 accumulation in
                            tensor memory, N <= 256); the weight gradients
                            stay FP32                                      */
} vs_ntex_config;

/* Offsets (in floats) of the seven parameter blocks and the total count.
 * Host only.  Errors: VS_ERR_INVALID_ARG for a config out of range. */
vs_status vs_ntex_layout(const vs_ntex_config* cfg, int64_t offsets[7], int64_t* total);

/* Workspace bytes for vs_ntex_forward / vs_ntex_backward on a tex_w x tex_h
 * texture (activations of up to 2^18 texels at a time).  Host only.  Its
 * first 4 bytes are a status word: zero the workspace once; with
 * tensor_cores = 1 a bounded wait that ran out writes 1 there (the layer's
 * outputs are then zero) and the call still returns. */
vs_status vs_ntex_workspace_size(const vs_ntex_config* cfg, int32_t tex_w, int32_t tex_h, size_t* bytes);

/* Evaluates the network at every texel centre and writes channels
 * [ch0, ch0 + C) of texels [tex_h, tex_w, pitch] (dtype 0 = float32,
 * 1 = float16, the renderer's SH storage).  FP32 arithmetic: the layers as
 * hand-written FP32 GEMMs with bias and ReLU fused, or on the tensor cores
 * in TF32 when cfg->tensor_cores = 1.
 * Errors: VS_ERR_INVALID_ARG (config, sizes, ch0 + C > pitch, NULL),
 * VS_ERR_WORKSPACE, VS_ERR_CUDA. */
vs_status vs_ntex_forward(vs_ctx* ctx, const vs_ntex_config* cfg, const float* params, int32_t tex_w, int32_t tex_h,
                          void* texels, int32_t dtype, int32_t pitch, int32_t ch0, void* workspace, size_t ws_bytes,
                          vs_stream_t stream);

/* Adjoint: given dL/d(texel values) (float32 [tex_h, tex_w, pitch], e.g.
 * from vs_render_backward), ADDS dL/d(params) into grads (same layout as
 * params; zero it first).  Recomputes the activations; hash-table gradients
 * use float atomics (summation order varies run to run).  Errors: as
 * vs_ntex_forward. */
vs_status vs_ntex_backward(vs_ctx* ctx, const vs_ntex_config* cfg, const float* params, int32_t tex_w, int32_t tex_h,
                           const float* grad_texels, int32_t pitch, int32_t ch0, float* grads, void* workspace,
                           size_t ws_bytes, vs_stream_t stream);

/* One Adam step (Kingma & Ba, bias-corrected) on n parameters in place:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * step >= 1.  Errors: VS_ERR_INVALID_ARG, VS_ERR_CUDA. */
vs_status vs_adam_step(vs_ctx* ctx, float* params, const float* grads, float* m, float* v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int32_t step, vs_stream_t stream);

/* --- allocation-free forward ------------------------------------------------- */

/* vs_render for callers that cannot allocate device memory at all, and so
 * cannot pass a workspace: a render loop that must not allocate once it is
 * running (allocation can block the loop and fragment memory), or a plug-in
 * inside a host framework that owns and pools every byte of device memory
 * and lends none out.  The paper has no counterpart; this is a deployment
 * convenience.
 *   Scratch: a fixed 16 MiB array in device memory that every GPU loading the
 *   library holds until the process exits.  One call needs about
 *   8 k H W + 16 sum(V) bytes plus a few KB (e.g. k = 3 shells at 512x512
 *   with up to 300k vertices); larger requests return VS_ERR_OVERFLOW with the
 *   needed size in vs_last_error(), before anything is enqueued.
 *   First calls: the first call on each device looks up the array's device
 *   address (cudaGetSymbolAddress), and the first render of each object --
 *   through this call or any other -- reads its vertex positions once with a
 *   blocking device-to-host copy (vs_load_shells).  Make both first calls
 *   before any stream capture, from ordinary host code (no CUDA call is
 *   allowed inside a stream callback).
 *   Sharing: every call uses the same array and leaves its contents there;
 *   each call re-initialises what must start at zero.  Calls that overlap on
 *   the GPU (e.g. on two streams of one device) race and corrupt each
 *   other's results: order them.  Device-side counters are not reported.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Arguments, outputs and errors as vs_render (without the workspace). */
vs_status vs_render_noalloc(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg,
                            float* out_rgba, int32_t* hits, uint32_t flags, vs_stream_t stream);

/* --- status and counters --------------------------------------------------------- */

typedef struct {
  vs_status device_status;   /* first error recorded on the device, or VS_OK  */
  uint64_t fragments;        /* (pixel, shell) pairs shaded (hits)            */
  uint64_t tris_front;       /* triangles rasterized (front-facing, valid)    */
  uint64_t tris_culled_back; /* back-facing or zero-area                       */
  uint64_t tris_culled_near; /* every vertex nearer than znear                */
  uint64_t tris_culled_guard;/* a vertex beyond +-32768 px                    */
  uint64_t tris_large;       /* rasterized cooperatively by a whole block     */
  uint64_t launches;         /* kernels enqueued by the calls (table uploads
                                included), as declared by the host side      */
  uint64_t tris_clipped;     /* one or two vertices nearer than znear: clipped
                                at the near plane, the rest rasterized       */
  int32_t kernel_class;      /* shading kernels of the last call: 1 + texel
                                class (0 any format, chosen per shell; 1 RGBA
                                F32; 2 + d SH F16 of degree d; 6 + d baked
                                bytes of degree d), + 16 for the variant with
                                near-plane clipping and per-layer buffers; 0
                                before any call                               */
  int32_t reserved;
} vs_stats;

/* Synchronizes `stream`, copies the counters accumulated in `workspace`
 * since the last reset into *out, and (reset != 0) zeroes them and the
 * device status.  The only call that synchronizes. */
vs_status vs_read_stats(void* workspace, vs_stream_t stream, int32_t reset, vs_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* VS_H_ */
