/*
 * ldni.h - C ABI of the GB300 LDNI library (libldni.so).
 *
 * Layered Depth-Normal Images (Wang & Chen): a closed triangle mesh is
 * sampled by the pixel-centre rays of three axis-aligned images; every ray
 * stores the ascending depths of its crossings with the surface, each with
 * the unit surface normal (Section 2, Definitions 1-3).  Solids are combined
 * per ray by 1D Boolean merges (Section 4.1).
 *
 * Conventions shared by every call
 *  - All data pointers are DEVICE pointers (CUDA global memory of the current
 *    device) unless a parameter says "host".  The caller owns every buffer;
 *    the library allocates nothing and keeps no device state between calls,
 *    with one exception: the static scratch array of ldni_boolean_static
 *    (4 MiB + 8.5 KiB on every GPU that loads the library, for res <= 1024;
 *    calls of that entry point that overlap on the GPU race on it).
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Host-side validation errors are returned
 *    immediately; conditions found on the device (capacity exceeded, odd
 *    rays, scan overflow) are written to the caller's device `info` block
 *    (ldni_info_t) and become visible once the stream has reached that point.
 *  - Grid (Definition 3): one cube [origin, origin + width]^3 shared by the
 *    three images; res x res pixels of pitch h = width / res.  Axis a in
 *    {0:x, 1:y, 2:z}; in-plane coordinates (u, v) = (y, z), (z, x), (x, y).
 *    Pixel (i, j), i along u and j along v, is row p = j * res + i; its ray
 *    passes through the pixel centre (Section 3) and runs along +a.
 *  - Depth is the world a-coordinate of a crossing, ascending along the ray
 *    (Definition 1 measures depth to the viewing plane; the two differ by a
 *    constant shift per image).
 *  - Return codes: LDNI_OK (0) or a negative LDNI_E* code (ldni_strerror).
 */
#ifndef LDNI_H
#define LDNI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------- */
#define LDNI_OK 0
#define LDNI_EINVAL (-1)          /* bad argument (null pointer, res <= 0, axis, op, ...) */
#define LDNI_EGRID_MISMATCH (-2)  /* Boolean operands on different grids (Section 4.1.1) */
#define LDNI_EODD (-3)            /* an input ray has an odd sample count (Definition 4) */
#define LDNI_ETOOLARGE (-4)       /* res or sample count beyond the int32 CSR range */
#define LDNI_EWORKSPACE (-5)      /* workspace smaller than the *_workspace_size query */
#define LDNI_ECUDA (-6)           /* a CUDA runtime call or launch failed */
#define LDNI_ETIMEOUT (-7)        /* a bounded device wait gave up */
#define LDNI_ERANGE (-8)          /* a vertex lies too far outside the cube to snap */
#define LDNI_ECAPACITY (-9)       /* output capacity smaller than the sample count */

/* ---- device-side status bits (ldni_info_t.status) ------------------- */
#define LDNI_ST_CAPACITY 1u       /* an output had more samples than capacity; extra dropped */
#define LDNI_ST_ODD 2u            /* an input or sampled ray had an odd count */
#define LDNI_ST_TOOLARGE 4u       /* a sample total exceeded 2^31 - 1 */
#define LDNI_ST_TIMEOUT 8u        /* a bounded device wait expired */
#define LDNI_ST_RANGE 16u         /* a vertex could not be snapped (outside +-2^24 units) */
#define LDNI_ST_INDEX 32u         /* a triangle referenced a vertex index outside [0, nv) */
#define LDNI_ST_EVENTS 64u        /* offsetting: a ray met more samples than one warp orders; left empty */
#define LDNI_ST_BOUNDS 128u       /* checked builds only (LDNI_CHECKS): a CSR or slab index outside its array
                                     was met and that access skipped; release builds never set it */

/* ---- modes and operations ------------------------------------------ */
#define LDNI_AXIS_X 0
#define LDNI_AXIS_Y 1
#define LDNI_AXIS_Z 2
#define LDNI_AXIS_ALL 3           /* the three images of Definition 3 in one call */
#define LDNI_MAX_IMAGES 8         /* images per ldni_boolean_many / ldni_volume_many call */

#define LDNI_MODE_EXACT2 0        /* exact two-pass: count, scan, fill, sort */
#define LDNI_MODE_LEARNED1 1      /* one pass into learned per-tile capacity, exact redo of overflow */
#define LDNI_MODE_BINNED2 2       /* exact two-pass with triangles binned to 16 x 16 pixel tiles */

#define LDNI_OP_UNION 0
#define LDNI_OP_INTER 1
#define LDNI_OP_DIFF 2

/* Fixed-point subpixel bits of the snap: pixel centre i sits at 256 i + 128. */
#define LDNI_SUBPIX_BITS 8

/* ---- data ---------------------------------------------------------- */

/* The cube shared by the three images (Definition 3). */
typedef struct {
    float origin[3]; /* minimum corner */
    float width;     /* cube edge length W > 0 */
    int32_t res;     /* pixels per image side, 1 .. 8192 */
} ldni_grid_t;

/* One layered depth-normal image in CSR form (Definitions 1-2).
 * Samples of ray p are rows offsets[p] .. offsets[p+1]-1, ascending by
 * (depth, tri_id).  SoA arrays, each `capacity` long; offsets has res*res+1
 * entries.  tri_id is the index of the sampled triangle ("accurate normal
 * sampling", Section 3 item 2); in a Boolean result bit 31 marks a sample
 * taken from the second operand.
 * Normals: with nrm8 == NULL, FP32 unit normals in nx, ny, nz.  With nrm8
 * set, approximate normals (Section 3 item 1): one 32-bit word per sample
 * holding three 8-bit codes (x in bits 0-7, y 8-15, z 16-23, the rest 0),
 * q = rint(fl32(fl32(n + 1) * 127.5)) half to even, clamped to [0, 255];
 * nx, ny, nz are then not used.  A decoded component is
 * fl32(fl32(q / 127.5) - 1), normalised (ldni_normals_decode8); inverting a
 * packed normal (Boolean difference) maps every q to 255 - q.  The inputs
 * and output of one call use one format; offsetting takes FP32 normals only. */
typedef struct {
    int32_t *offsets;
    float *depth;
    float *nx;
    float *ny;
    float *nz;
    int32_t *tri_id;
    int64_t capacity; /* host value: length of the five sample arrays */
    uint32_t *nrm8;   /* NULL, or packed 8-bit normals (capacity words) in place of nx, ny, nz */
} ldni_layers_t;

/* Device block a call reports into (caller-owned, device memory).
 * n[a]  : number of samples the call produced (or needed) for image a
 *         (a = the axis, also for single-axis calls); Booleans use n[0].
 * status: OR of LDNI_ST_* bits; the library ORs into it, the caller clears. */
typedef struct {
    int64_t n[3];
    uint32_t status;
    uint32_t odd_rays; /* rays with an odd count seen by the call */
} ldni_info_t;

/* The per-tile capacity network of the one-pass sampler: 12 tile features
 * -> 64 -> 64 -> 64 -> 1 with ReLU on the hidden layers.  Weights are BF16,
 * row-major [out][in], layers concatenated: W0 [64][12] at 0, W1 [64][64] at
 * 768, W2 [64][64] at 4864, W3 [1][64] at 8960 (9024 values).  Biases are
 * FP32: b0[64] at 0, b1[64] at 64, b2[64] at 128, b3[1] at 192 (193 values).
 * Output y predicts log1p(largest ray count in the tile); the tile's layer
 * capacity is k = ceil(expm1(y) * (1 + margin)) rounded up to even, in
 * [2, 64]. */
typedef struct {
    const uint16_t *w; /* device, 9024 BF16 weights */
    const float *b;    /* device, 193 FP32 biases */
    float margin;
} ldni_mlp_t;

#define LDNI_MLP_IN 12
#define LDNI_MLP_WEIGHTS 9024
#define LDNI_MLP_BIASES 193
#define LDNI_TILE_RAYS 4096 /* a tile = 4096 consecutive rays of one image (CSR order) */

/* ---- helpers ------------------------------------------------------- */

/* Human-readable text for a return code (static storage, never NULL). */
const char *ldni_strerror(int code);

/* Text of the CUDA error behind the calling thread's most recent
 * LDNI_ECUDA (static storage, never NULL; "no CUDA error" before any). */
const char *ldni_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int ldni_version(void);

/* Grid from a host bbox[6] = {min x, min y, min z, max x, max y, max z}:
 * origin = bbox min, width = largest extent (the caller pads the box; the
 * paper uses a working envelope slightly larger than the model, Section 3). */
int ldni_grid_from_bbox(const float *bbox_host, int32_t res, ldni_grid_t *grid_host);

/* One mesh of a batch (ldni_sample_batch): its three images x, y, z on its
 * own grid.  The array of items lives in DEVICE memory for the kernels; the
 * same values are passed as a host copy for validation and sizing. */
typedef struct {
    const float *verts;   /* device float[nv][3] */
    const int32_t *tris;  /* device int32[nt][3] */
    int64_t nv;
    int64_t nt;
    ldni_grid_t grid;
    int32_t pad_;         /* keeps out[] 8-byte aligned */
    ldni_layers_t out[3]; /* device buffers of the three images */
} ldni_batch_item_t;

/* ---- sampling (Section 3; Definitions 1-4; Remark 1) ---------------- */

/* Bytes of device workspace ldni_sample / ldni_sample_count need for a mesh
 * of nt triangles at grid->res and the given axis (0..2 or LDNI_AXIS_ALL). */
int ldni_sample_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis, size_t *bytes_host);

/*
 * Sample a closed triangle mesh into one or three LDNIs.
 *   verts  : device float[nv][3], world coordinates.
 *   tris   : device int32[nt][3], vertex indices, outward winding.
 *   grid   : host pointer to the cube.
 *   axis   : 0, 1, 2, or LDNI_AXIS_ALL (out then points to 3 layers x, y, z).
 *   mode   : LDNI_MODE_EXACT2 - count pass, scan, fill pass, per-ray sort;
 *            the paper's stencil-counted multi-pass rendering (Section 3,
 *            Appendix A) restated for CUDA; or LDNI_MODE_BINNED2 - the same
 *            passes tile by tile (ldni_sample_binned_count, needs the binned
 *            workspace), identical output.
 *   out    : host pointer to 1 or 3 ldni_layers_t with caller buffers.
 *   info   : device ldni_info_t; n[a] receives the sample count of image a.
 *   ws     : device workspace of at least ldni_sample_workspace_size bytes.
 * A ray crosses a triangle iff the ray's fixed-point pixel centre lies in the
 * triangle's snapped projection under the top-left rule, so a shared
 * non-silhouette edge is crossed once and a silhouette edge 0 or 2 times
 * (Remark 1); faces parallel to the ray are not sampled (Definition 1 note).
 * If a count exceeds out[a].capacity the extra samples are dropped, bit
 * LDNI_ST_CAPACITY is set and info->n[a] holds the size needed.  An odd ray
 * (a mesh that is not closed or self-intersects, Remark 2) sets LDNI_ST_ODD.
 */
int ldni_sample(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                int32_t axis, int32_t mode, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                void *stream);

/* First half of ldni_sample (count pass + scan): writes out[a].offsets and
 * info->n[a] so that a caller can size the sample arrays exactly, then calls
 * ldni_sample_fill with the same workspace.  Only offsets of `out` are used. */
int ldni_sample_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                      int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                      void *stream);

/* Second half of ldni_sample (fill pass + per-ray sort + CSR write) after
 * ldni_sample_count on the same workspace, same inputs and same offsets. */
int ldni_sample_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                     int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                     void *stream);

/* ---- exact two-pass sampling with tile binning ------------------------- */

/* Bytes of device workspace of ldni_sample with LDNI_MODE_BINNED2 and of its
 * two halves below; LDNI_ETOOLARGE beyond 2^31 / 16 triangles. */
int ldni_sample_binned_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis, size_t *bytes_host);

/*
 * ldni_sample's result (identical bits) with a different traversal, for
 * meshes whose triangles cover many pixels or whose rays hold many layers:
 * a counting sort bins every (triangle, image) pair to the 16 x 16 pixel
 * tiles its pixel box touches, and one block per tile stages the exact
 * setup of its triangles (snapped, oriented edge functions; Remark 1's
 * top-left rule) in shared memory while every thread - one pixel centre -
 * tests them all.  A pixel counts its crossings in a register and writes them
 * to its own slots, with no atomic per crossing.  Pairs whose box touches
 * more than 16 tiles take the direct form's big-triangle path.  Both halves
 * take the same arguments as ldni_sample_count / ldni_sample_fill, with the
 * binned workspace; call count, size the arrays from info->n, then fill.
 */
int ldni_sample_binned_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                             const ldni_grid_t *grid, int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws,
                             size_t ws_bytes, void *stream);
int ldni_sample_binned_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                            int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                            void *stream);

/* ---- launch tuning ---------------------------------------------------- */

/* Launch-shape knobs.  They change speed only, never a result: every setting
 * produces the same bits.  The values are process-wide host state, read when
 * a call launches its kernels (a captured CUDA graph keeps the shapes it was
 * captured with).  Setting them while another thread is launching is a race
 * on the host. */
typedef struct {
    int32_t bool_tile_rays;      /* rays per Boolean block: 256, 512, 1024 or 2048 */
    int32_t bool_stage_samples;  /* samples of a Boolean tile staged in shared memory,
                                    0 (merge from global memory) .. 16384 */
    int32_t tri_blocks_per_sm;   /* grid of the per-triangle sampling passes, 1 .. 64 */
    int32_t bool_split;          /* Boolean as one launch (0), as count and write launches (1),
                                    or chosen by image size (-1) */
} ldni_tuning_t;

/* Current knobs (defaults: 512, 4096, 16, -1). */
int ldni_get_tuning(ldni_tuning_t *tuning_host);
/* Replace the knobs; LDNI_EINVAL (and no change) when a value is out of range.
 * NULL restores the defaults. */
int ldni_set_tuning(const ldni_tuning_t *tuning_host);

/* ---- bounded device waits (no counterpart in the paper) ------------------ */

/* Polls a bounded device wait (the decoupled look-back of the one-launch
 * scans, Booleans and batches) makes before it gives up; it then records
 * LDNI_ST_TIMEOUT in the call's info block and the kernel ends, so no kernel
 * of the library waits forever.  Process-wide host state read when a call
 * launches (a captured CUDA graph keeps the value it was captured with).
 * polls 0 restores the default (2^22); negative is LDNI_EINVAL. */
int ldni_set_wait_limit(int32_t polls);
int32_t ldni_get_wait_limit(void);

/* Self-test of the timeout path: one warp runs the bounded wait, with the
 * current limit, on a word that nothing sets; info->status (device) gains
 * LDNI_ST_TIMEOUT once the stream reaches that point.  Nothing else is
 * touched, and the device stays usable. */
int ldni_wait_selftest(ldni_info_t *info, void *stream);

/* 1 when the loaded library is a checked build (compiled with LDNI_CHECKS:
 * CSR and slab ranges are tested before they are touched and reported as
 * LDNI_ST_BOUNDS), 0 for a release build.  A debugging aid in place of a
 * memory checker; no GPU needed. */
int32_t ldni_build_checked(void);

/* ---- batches ------------------------------------------------------------ */

/* Workspace bytes for ldni_sample_batch over items_host[count]. */
int ldni_sample_batch_workspace_size(const ldni_batch_item_t *items_host, int32_t count, size_t *bytes_host);

/*
 * ldni_sample (exact two-pass, all three images) for `count` meshes of any
 * sizes and resolutions with one launch per stage for the whole batch:
 * count, big-triangle count, scan, fill, big-triangle fill, per-ray sort.
 * Paper's use: repeated solid modelling operations work on LDNIs of many
 * solids on one grid (Section 1; Section 4.1.1 chains; Section 4.2 sphere
 * unions).  items_dev: device array of count items (read by the kernels);
 * items_host: the same items on the host (validation, workspace carving).
 * infos: device ldni_info_t[count], one per item (n[a] per image); cleared
 * by the call itself, so replays of a captured call start from zero.  The
 * output is bit-identical to sampling each item alone.  Makes no host
 * synchronisation, so a call can be captured in a CUDA graph as long as the
 * item array and workspace outlive the graph.
 */
int ldni_sample_batch(const ldni_batch_item_t *items_dev, const ldni_batch_item_t *items_host, int32_t count,
                      ldni_info_t *infos, void *ws, size_t ws_bytes, void *stream);

/* ---- one-pass sampling with learned capacity ------------------------------ */

/* Workspace bytes for ldni_sample_learned with a slab of slab_samples slots. */
int ldni_sample_learned_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis, int64_t slab_samples,
                                       size_t *bytes_host);

/*
 * The LDNIs of ldni_sample (identical output) from ONE traversal of the mesh
 * instead of the count-then-fill pair.  The paper's count pass exists to size
 * each pixel's layer list before the layers are captured (Section 3: the
 * stencil pass, then passes 2..n_max); here a network predicts, per tile of
 * LDNI_TILE_RAYS rays, the largest layer count k_t of its rays from features
 * of a 1-in-feature_stride triangle subsample taken as runs of 8
 * consecutive triangles (count, projected area, mean |n_a|, depth
 * histogram).  Every ray of tile t gets k_t slots of a slab in
 * the workspace; a crossing that does not fit marks its tile, and marked
 * tiles are filled again by the exact method, so the output never depends on
 * the prediction.
 *   mlp          : host pointer to the network, or NULL to give every tile
 *                  fixed_layers slots (the baseline without the network).
 *   slab_samples : slab slots in the workspace; tiles beyond it are redone.
 *   overflow_tiles: optional device int32, receives the number of redone tiles.
 * Other arguments, output and status as ldni_sample.
 */
int ldni_sample_learned(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                        int32_t axis, const ldni_mlp_t *mlp, int32_t fixed_layers, int32_t feature_stride,
                        int64_t slab_samples, ldni_layers_t *out, ldni_info_t *info, int32_t *overflow_tiles, void *ws,
                        size_t ws_bytes, void *stream);

/* Tile features as the network sees them: raw = device scratch of
 * naxes * ntiles * 11 floats (cleared by the call); X = device output of
 * naxes * ntiles * 12 floats, rows image-major then tile.  ntiles =
 * ceil(res^2 / LDNI_TILE_RAYS). */
int ldni_tile_features(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                       int32_t axis, int32_t feature_stride, float *raw, float *X, void *stream);

/* Training target per tile of one exact LDNI: label[t] = log1p(largest ray
 * count of tile t), from its CSR offsets (device, res*res+1). */
int ldni_tile_labels(const int32_t *offsets, int32_t res, float *label, void *stream);

/* Network outputs y[n] (device) for feature rows X[n][12] (device). */
int ldni_mlp_forward(const ldni_mlp_t *mlp, const float *X, int64_t n, float *y, void *stream);

/* Workspace bytes for ldni_mlp_train_step on n rows. */
int ldni_mlp_train_workspace_size(int64_t n, size_t *bytes_host);

/*
 * One Adam step on the capacity network, all on the device.
 *   master_w [9024], b [193]: FP32 parameters, updated in place;
 *   w_bf16 [9024]: refreshed BF16 copy used by the forward pass;
 *   m, v [9024 + 193]: Adam moments (weights first, then biases);
 *   X [n][12], label [n]: training rows;
 *   loss: device float, receives the loss before the update;
 *   grad: optional device [9024 + 193], receives the gradient.
 * Loss = mean over rows of w * (y - label)^2 with w = under_weight where
 * y < label (a predicted capacity below the truth costs a redo) and 1
 * otherwise.  Forward with the BF16 weights, FP32 everywhere else.
 */
int ldni_mlp_train_step(float *master_w, float *b, uint16_t *w_bf16, float *m, float *v, const float *X,
                        const float *label, int64_t n, float lr, int32_t step, float under_weight, float *loss,
                        float *grad, void *ws, size_t ws_bytes, void *stream);

/* ---- Boolean (Section 4.1, small-interval removal Section 4.1.1) ----- */

/* Workspace bytes for ldni_boolean at resolution res. */
int ldni_boolean_workspace_size(int32_t res, size_t *bytes_host);

/*
 * out = A op B (Section 4.1).  A, B, out: host pointers to layers with device
 * buffers; grid_a, grid_b: host pointers to the operands' grids, which must
 * be identical (same origin and sampling rate, Section 4.1.1), else
 * LDNI_EGRID_MISMATCH.  Per ray the result is the boundary of
 * {t : op(in_A(t), in_B(t))} where in_X(t) means an odd number of X samples
 * lie below t; equal depths of A and B are one event; an emitted sample is
 * copied from A when A's state flips there, else from B (normal inverted for
 * LDNI_OP_DIFF; tri_id | 0x80000000).  Then every solid interval thinner than
 * eps (FP32 difference, strict <) is removed.  out->capacity >=
 * A.capacity + B.capacity always suffices; extra samples beyond capacity are
 * dropped (LDNI_ST_CAPACITY).  info->n[0] = output count; odd input rays set
 * LDNI_ST_ODD.
 */
int ldni_boolean(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B, const ldni_grid_t *grid_b,
                 int32_t op, float eps, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                 void *stream);

/* Workspace bytes for ldni_boolean_many of `count` images at resolution res. */
int ldni_boolean_many_workspace_size(int32_t res, int32_t count, size_t *bytes_host);

/*
 * ldni_boolean for `count` (1 .. LDNI_MAX_IMAGES) image pairs on one grid in
 * one set of launches: out[j] = A[j] op B[j], typically the three images of
 * two solids (Definition 3).  A, B, out: host arrays of count layers; infos:
 * device array of count ldni_info_t.  Each result is the one ldni_boolean
 * gives for that pair.
 * vols: NULL, or device double[count] receiving the volume of each result
 * as ldni_volume defines it (h^2 times the summed inside lengths), summed
 * while the result is written (double-float, fixed order; equal to
 * ldni_volume's value to about 1e-13 relative).
 */
int ldni_boolean_many(int32_t count, const ldni_layers_t *A, const ldni_layers_t *B, const ldni_grid_t *grid,
                      int32_t op, float eps, ldni_layers_t *out, ldni_info_t *infos, double *vols, void *ws,
                      size_t ws_bytes, void *stream);

/*
 * ldni_boolean without a workspace argument, for callers that cannot
 * allocate device memory where they need a Boolean (code that is handed only
 * input and output buffers because another framework owns the device
 * allocator, or a loop where an allocation would synchronise the device).
 * The paper has no counterpart; this is a deployment variant.
 * Scratch: one static device array of 4 MiB + 8.5 KiB in the library, held by
 * every GPU that loads the library until the process exits.  Limit: res <=
 * 1024, else LDNI_ETOOLARGE.  The first call in a CUDA context (the
 * device's primary context, another context of that device, or the primary
 * context made again after cudaDeviceReset) looks up that array's device
 * address in the context (cudaGetSymbolAddress) and caches it per context;
 * make that first call before any stream capture.  No call allocates or
 * frees memory.
 * All calls share the array: calls whose work overlaps on the GPU (two
 * streams, or two host threads) race and corrupt each other's results;
 * serialise them.  Each call writes every scratch word it reads, so the
 * previous call's leftovers do not matter.  Same arguments, semantics and
 * results as ldni_boolean otherwise.
 */
int ldni_boolean_static(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B,
                        const ldni_grid_t *grid_b, int32_t op, float eps, ldni_layers_t *out, ldni_info_t *info,
                        void *stream);

/* ---- chains of unions (Sections 4.1.1 and 4.2) -------------------------- */

/* Workspace bytes for ldni_union_chain of nimg (1 .. 3) images at res. */
int ldni_union_chain_workspace_size(int32_t res, int32_t nimg, size_t *bytes_host);

/*
 * out[j] = P[j][0] u P[j][1] u ... u P[j][count-1] for each image j, all on
 * one grid: the repeated union of offsetting and sweeps (Section 4.2) and of
 * any chain of Booleans on one grid (Section 4.1.1).  The result is the one
 * the step-by-step chain of ldni_boolean calls gives,
 *   acc = P[j][0];  acc = ldni_boolean(acc, P[j][k], LDNI_OP_UNION, eps)  (k = 1 ..),
 * bit for bit: small-interval removal after every step, the accumulated
 * sample kept where both flip at one depth, and tri_id bit 31 on every
 * sample that entered through a part k >= 1.  Each ray carries its own
 * accumulated samples from step to step (two passes over the rays and the
 * CSR scan; no intermediate image is written).
 *   parts_dev  : DEVICE array of nimg * count layers, image-major (part k of
 *                image j at j * count + k), read by the kernels;
 *   parts_host : the same array on the host (validation);
 *   out        : host array of nimg layers with device buffers; the inputs
 *                and the output share one normal format;
 *   info       : device; n[j] = samples image j of the result needs (beyond
 *                out[j].capacity they are dropped, LDNI_ST_CAPACITY).
 * A ray whose accumulated result would need more than 64 samples at some
 * step is left empty and reported (LDNI_ST_EVENTS); odd input rays set
 * LDNI_ST_ODD.  No host synchronisation (capturable in a CUDA graph while the
 * parts array and workspace outlive the graph).
 */
int ldni_union_chain(const ldni_layers_t *parts_dev, const ldni_layers_t *parts_host, int32_t count, int32_t nimg,
                     const ldni_grid_t *grid, float eps, ldni_layers_t *out, ldni_info_t *info, void *ws,
                     size_t ws_bytes, void *stream);

/* ---- volume ----------------------------------------------------------- */

/* Workspace bytes for ldni_volume at resolution res. */
int ldni_volume_workspace_size(int32_t res, size_t *bytes_host);

/*
 * Enclosed volume seen by one LDNI: h^2 * sum over rays of
 * (d[2k+1] - d[2k]) - the odd-to-even ranges are inside (Section 2, after
 * Proposition 1).  vol: device double, written.  Deterministic (fixed
 * reduction order).  Odd rays set LDNI_ST_ODD and are skipped.
 */
int ldni_volume(const ldni_layers_t *L, const ldni_grid_t *grid, double *vol, ldni_info_t *info, void *ws,
                size_t ws_bytes, void *stream);

/* Workspace bytes for ldni_volume_many of `count` images at resolution res. */
int ldni_volume_many_workspace_size(int32_t res, int32_t count, size_t *bytes_host);

/* ldni_volume of `count` (1 .. LDNI_MAX_IMAGES) images of one grid in one
 * launch.  L: host array of count layers; vols: device double[count];
 * infos: device ldni_info_t[count]. */
int ldni_volume_many(int32_t count, const ldni_layers_t *L, const ldni_grid_t *grid, double *vols, ldni_info_t *infos,
                     void *ws, size_t ws_bytes, void *stream);

/* ---- approximate normals (Section 3 item 1) ---------------------------- */

/* Packed 8-bit codes of n FP32 normals (device arrays; the ldni_layers_t
 * codec: q = rint(fl32(fl32(c + 1) * 127.5)) half to even, clamped to
 * [0, 255], x in bits 0-7, y 8-15, z 16-23). */
int ldni_normals_encode8(const float *nx, const float *ny, const float *nz, int64_t n, uint32_t *w, void *stream);

/* Unit FP32 normals from n packed words: c = fl32(fl32(q / 127.5) - 1) per
 * component, divided by sqrt(fl32(fl32(cx^2 + cy^2) + cz^2)), each operation
 * rounded to nearest. */
int ldni_normals_decode8(const uint32_t *w, int64_t n, float *nx, float *ny, float *nz, void *stream);

/* ---- contouring, Steps 2-3 (Section 5.1) ------------------------------- */

/* One cell (i, j, k) of the node grid that yields a vertex: its corners are
 * nodes (i + di, j + dj, k + dk), corner c = di + 2 dj + 4 dk. */
typedef struct {
    int64_t cell;    /* i + (res - 1) (j + (res - 1) k) */
    uint32_t labels; /* 4 bits per corner c at bit 4c: its cluster (= vertex), 0xF inside */
    uint32_t npts;   /* 8 bits per vertex g at bit 8g: Hermite points fitted (saturating at 255) */
    int32_t nvert;   /* 1 .. 4 */
    int32_t pad_;
    float v[12];     /* vertex g at v[3g], v[3g + 1], v[3g + 2] (x, y, z) */
} ldni_cell_t;

/* Workspace bytes for ldni_contour_cells at resolution res (2 .. 2048) with
 * room for max_active cells next to an edge that holds a sample or joins
 * nodes of different sign. */
int ldni_contour_workspace_size(int32_t res, int64_t max_active, size_t *bytes_host);

/*
 * Steps 2 and 3 of the contouring of Section 5.1.  The edge (t, t + 1)
 * along axis a between grid nodes lies on the ray of image a through its two
 * other node indices and holds the samples with c_a(t) <= d < c_a(t + 1)
 * (node coordinates as in ldni_classify_nodes).  Edge types follow the end
 * signs (inside: from ldni_classify_nodes) and the samples: intersect
 * (signs differ, samples), none-intersect, empty (same sign, none),
 * complex.  Rule 1: a complex edge keeps its first and last samples; Rule
 * 2: an intersect edge keeps, of the samples whose normal's a-component
 * points from the inside end to the outside end (all samples if none), the
 * one nearest the edge's midpoint (the earlier on a tie).  In every cell the
 * outside corners joined by empty edges form clusters, numbered by their
 * lowest corner; a cluster takes the kept sample of each intersect edge at
 * one of its corners and, of each complex edge between outside corners, the
 * sample nearer each corner (a single sample goes to the nearer corner).
 * Each cluster that meets an intersect, none-intersect or complex edge gets
 * a vertex at x = m + (A^T A)^+ (A^T b - A^T A m) over its Hermite points p
 * (rows of A: the normals n; b = n . p; m: the points' mean), eigenvalues of
 * A^T A below 0.01 of the largest dropped, in FP64; with no points, at the
 * mean of its corners (npts 0).
 *   L: host array of the three images x, y, z (FP32 normals); inside: the
 *   node bits; cells: device array of `capacity` records, written in
 *   ascending cell order.  info->n[0] = cells with a vertex; beyond capacity
 *   they are dropped (LDNI_ST_CAPACITY); more than max_active active cells
 *   also set LDNI_ST_CAPACITY.  No host synchronisation.
 */
int ldni_contour_cells(const ldni_layers_t *L, const ldni_grid_t *grid, const uint32_t *inside, int64_t max_active,
                       ldni_cell_t *cells, int64_t capacity, ldni_info_t *info, void *ws, size_t ws_bytes,
                       void *stream);

/* ---- offsetting (Section 4.2) ------------------------------------------ */

/* Workspace bytes for ldni_offset of a solid whose three images hold n[0],
 * n[1], n[2] samples (host array), at resolution res, radius r and cube
 * width `width`.  The sphere lists grow with (r / h)^2 per sample;
 * LDNI_ETOOLARGE when they would pass 2^31 - 1 entries or the samples 2^30. */
int ldni_offset_workspace_size(const int64_t *n, int32_t res, float r, float width, size_t *bytes_host);

/*
 * Offset of the solid H given by its three LDNIs (Section 4.2): H united
 * with (inner = 1: minus) one sphere of radius r about every sample of H,
 * each sphere represented by its LDNIs on H's grid, then small-interval
 * removal with eps (FP32 difference, strict <) applied once.
 * Sample (i, j, d) of image a sits at the point with a-coordinate d and
 * in-plane coordinates c_u(i), c_v(j), c(t) = fl32(o + fl32((t + 1/2) h)),
 * h = fl32(width / res); spheres are numbered in sample order (image x, y,
 * z, each in CSR order).  Sphere s about C meets the ray (P_u, P_v) of image
 * b iff q < fl32(r r), q = fl32(fl32(du du) + fl32(dv dv)),
 * du = fl32(P_u - C_u), dv = fl32(P_v - C_v); its samples are
 * fl32(C_b -+ sqrt(fl32(r r - q))) with outward normals (du, dv, -+t) / r
 * (componentwise FP32), id s | 0x80000000.  The result equals uniting
 * (subtracting) the spheres one by one in that order with the Boolean of
 * Section 4.1: where the result changes state, its sample is taken from the
 * first of H, sphere 0, sphere 1, ... that changes state there; normals of
 * subtracted spheres are inverted.
 * H, out: host arrays of 3 layers (image x, y, z) with device buffers on one
 * grid; n: host int64[3], the samples of H's images.  info: device, n[b] =
 * samples image b of the result needs; beyond out[b].capacity samples are
 * dropped (LDNI_ST_CAPACITY) while the offsets are still complete.  A ray
 * that meets more than 512 samples (H's plus two per sphere that can change
 * it) is left empty with LDNI_ST_EVENTS.  Odd input rays set LDNI_ST_ODD.
 */
int ldni_offset(const ldni_layers_t *H, const int64_t *n, const ldni_grid_t *grid, float r, int32_t inner, float eps,
                ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes, void *stream);

/* ---- grid-node classification (Section 5.1, Step 1) -------------------- */

/* Workspace bytes for ldni_classify_nodes at resolution res (<= 4096):
 * three bit volumes of res^2 * ceil(res / 32) words. */
int ldni_classify_nodes_workspace_size(int32_t res, size_t *bytes_host);

/*
 * Inside/outside status of the res^3 grid nodes where the rays of the three
 * images meet (Definition 3).  Node (i, j, k) lies at (c_x(i), c_y(j),
 * c_z(k)), c_a(t) = fl32(o_a + fl32((t + 1/2) * h)), h = fl32(width / res).
 * Image a puts the node inside when an odd number of the samples of its ray
 * through the node are strictly below c_a; the node is inside when at least
 * two images do (Section 5.1, Step 1).
 *   L      : host array of the three images x, y, z of one solid on `grid`.
 *   inside : device uint32[res][res][ceil(res/32)], bit (i % 32) of word
 *            [k][j][i / 32] = node (i, j, k); bits past res are 0.
 * Odd rays set LDNI_ST_ODD in info.
 */
int ldni_classify_nodes(const ldni_layers_t *L, const ldni_grid_t *grid, uint32_t *inside, ldni_info_t *info,
                        void *ws, size_t ws_bytes, void *stream);

/* ---- adjoint of depth and volume ---------------------------------------- */

/*
 * Vector-Jacobian product of the sample depths of one LDNI with respect to
 * the mesh vertices.  A sample of ray (u, v) on triangle t lies on t's plane,
 * d = sum_k lambda_k a_k (lambda: barycentrics of (u, v) in t's unsnapped
 * projection), so d(d)/d(V_j) = lambda_j n / n_a with n t's face normal.  The
 * set of crossings is held fixed (no boundary terms).
 *   L          : an LDNI sampled from exactly this mesh (tri_id = triangle),
 *                image `axis` of `grid`.
 *   grad_depth : device float[L.capacity], dLoss/d(depth) per sample.
 *   grad_verts : device float[nv][3], ACCUMULATED into (FP32 atomics).
 */
int ldni_depth_vjp(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                   int32_t axis, const ldni_layers_t *L, const float *grad_depth, float *grad_verts, ldni_info_t *info,
                   void *stream);

/*
 * Gradient of the LDNI volume h^2 sum_rays sum_k (d_{2k+1} - d_{2k}) (the
 * odd-to-even ranges are inside, Section 2 after Proposition 1) with respect
 * to the vertices, scaled by grad_volume (host) and ACCUMULATED into
 * grad_verts (device float[nv][3]).  Same fixed-crossing-set reading as
 * ldni_depth_vjp.
 */
int ldni_volume_grad(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                     int32_t axis, const ldni_layers_t *L, double grad_volume, float *grad_verts, ldni_info_t *info,
                     void *stream);

/* ---- instrumentation (no counterpart in the paper) ------------------- */

/* Number of kernels this process has launched through the library. */
uint64_t ldni_launch_count(void);

/*
 * Optional per-kernel timing.  begin_events / end_events: host arrays of
 * `capacity` cudaEvent_t (created by the caller); kernel_ids: optional host
 * int32 array of the same length that receives each record's kernel id.
 * From now on every launch of a kernel whose id equals `filter` (0 = every
 * kernel) records begin_events[k] before and end_events[k] after it on its
 * stream, k cycling through 0..capacity-1.  capacity 0 turns recording off.
 * Host state of the process, not thread-safe; for benchmarks only.
 */
int ldni_profile_set(void **begin_events, void **end_events, int32_t *kernel_ids, int32_t capacity, int32_t filter);

/* Records made since the last ldni_profile_set. */
int64_t ldni_profile_recorded(void);

/* Name of a kernel id (1 count_tri, 2 count_big, 4 scan_tiles, 5 scan,
 * 6 fill_tri, 7 fill_big, 8 sort_rays, 9 bool_count and 10 bool_write (the
 * count and write passes of the two-launch Boolean), 11 volume, 13 boolean, 14 features,
 * 15 capacity, 16 layout, 17 onepass, 18 onepass_big, 19 redo, 20 gather,
 * 21 mlp, 22 adjoint, 23 batch, 24 nodes, 25 order, 26 offset, 27 normals8, 28 contour, 29 chain, 30 bin,
 * 31 tile; 3, 12 and 32 are retired ids, named "unused"). */
const char *ldni_kernel_name(int32_t id);

#ifdef __cplusplus
}
#endif
#endif /* LDNI_H */
