/*
 * rad.h -- C ABI of the GB300 (sm_103a) shape-feature library.
 *
 * The library computes the 3D shape features that PyRadiomics-cuda
 * accelerates (arXiv 2510.02894, Sec. 2 "PyRadiomics-cuda design"): a
 * marching-cubes triangle mesh of a region-of-interest mask with its
 * MeshVolume and SurfaceArea (first step, Sec. 2), then the maximum 3D
 * diameter and the three planar diameters over the mesh vertices (second
 * step, Sec. 2 "Parallel diameter calculation"), plus VoxelVolume.
 *
 * Conventions (all entry points):
 *   - A mask is C-order [nz][ny][nx], x fastest; dims = {nx, ny, nz};
 *     spacing = {sx, sy, sz} in mm (finite, > 0).  1 <= n_k <= 16383.
 *   - The mask is implicitly padded with one outside voxel on every side.
 *     A uint8 voxel is inside iff != 0; a float32 voxel iff > 0.5.
 *   - Vertices: one per grid edge whose endpoints differ in inside-ness,
 *     ids in canonical (z, y, x, axis) order of the edge's lower endpoint.
 *     A vertex is stored as doubled index coordinates
 *     (2 g_k + [k == axis]), int16 x 3, plus (soft maps) the iso crossing
 *     parameter t from the lower endpoint, t = (0.5 - v0) / (v1 - v0).
 *   - Triangles: int32 x 3 vertex ids, wound counter-clockwise seen from
 *     outside.  Loops of 4+ vertices take the admissible triangulation of
 *     minimum area (ties: larger enclosed volume, then the smallest sorted
 *     list of canonical id triples).
 *   - Diameters: d2 = ((Dx Dx + Dy Dy) + Dz Dz), D_k = (u_ik - u_jk) s_k in
 *     FP64 (u = index position), D = sqrt(max d2); the argmax pair is the
 *     smallest (i, j), i < j, attaining the maximum.  Slice = pairs of equal
 *     z, Column = equal y, Row = equal x.  No pair: 0 and (-1, -1).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device
 *     pointers must be device-accessible from the current device.
 *   - No exception crosses the ABI.  Every call returns a rad_status; the
 *     text of the last error of the calling thread is rad_last_error().
 *   - Calls that return results to the host synchronise `stream`.
 */
#ifndef RAD_H_
#define RAD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RAD_OK = 0,
  RAD_ERR_INVALID_ARG = 1, /* bad pointer, size or spacing; nothing launched */
  RAD_ERR_CUDA = 2,        /* a CUDA runtime call failed (text in rad_last_error) */
  RAD_ERR_CAPACITY = 3,    /* an output pool was too small; the needed sizes are reported */
  RAD_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  RAD_ERR_OOM = 5,         /* device allocation failed */
  RAD_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} rad_status;

/* Features of one mask (names as in PyRadiomics' Shape class).
 * The derived features follow the standard Shape-class definitions, with V =
 * MeshVolume and A = SurfaceArea:
 *   Sphericity = (36 pi V^2)^(1/3) / A, SurfaceVolumeRatio = A / V,
 *   Compactness1 = V / (sqrt(pi) A^(3/2)), Compactness2 = 36 pi V^2 / A^3,
 *   SphericalDisproportion = A / (36 pi V^2)^(1/3);
 * and, from the eigenvalues l1 >= l2 >= l3 of the covariance (1/N) of the
 * physical coordinates of the N inside voxel centres:
 *   Major/Minor/LeastAxisLength = 4 sqrt(l1), 4 sqrt(l2), 4 sqrt(l3),
 *   Elongation = sqrt(l2 / l1), Flatness = sqrt(l3 / l1).
 * A feature with a zero denominator is 0. */
typedef struct {
  double MeshVolume, SurfaceArea, VoxelVolume;
  double Maximum3DDiameter, Maximum2DDiameterSlice, Maximum2DDiameterColumn, Maximum2DDiameterRow;
  int64_t n_vertices, n_triangles, n_voxels;
  int32_t argmax3d[2], argmax_slice[2], argmax_column[2], argmax_row[2];
  int32_t status; /* rad_status of this mask (batched calls) */
  int32_t _pad;
  double Sphericity, SurfaceVolumeRatio, Compactness1, Compactness2, SphericalDisproportion;
  double MajorAxisLength, MinorAxisLength, LeastAxisLength, Elongation, Flatness;
} rad_features_t;

/* A mesh on the device.  Zero-initialise before the first rad_mesh(); the
 * library owns the buffers (grown as needed, reused by later calls) and
 * frees them in rad_mesh_free().  The pointers stay valid until the next
 * rad_mesh()/rad_soft_mesh() or rad_mesh_free() on the same struct. */
typedef struct {
  int64_t n_vertices, n_triangles, n_voxels;
  int16_t* vtx_idx2; /* device, n_vertices x 3: doubled index coordinates */
  double* vtx_t;     /* device, n_vertices: crossing parameter (soft meshes; NULL for masks) */
  int32_t* tri;      /* device, n_triangles x 3 */
  double mesh_volume, surface_area;
  int64_t dims[3];
  double spacing[3];
  int32_t soft;
  int32_t _pad;
  void* _priv; /* library-owned state */
} rad_mesh_t;

/* Tuning knobs of the diameter kernels (see rad_set_tuning). */
typedef struct {
  int32_t tile;        /* vertices per tile: 64, 128 or 256 */
  int32_t threads;     /* threads per CTA of the pair kernel: 64 or 128, also 256 with
                          tiles of 128 vertices */
  int32_t ctas_per_sm; /* persistent CTAs per SM for the pair kernel: 1..16 */
  int32_t cell_shift;  /* spatial cell edge = 2^cell_shift doubled-index units (2..7) */
} rad_tuning_t;

/* ---- single mask --------------------------------------------------------- */

/* Marching cubes (Sec. 2, "Marching cubes fused parallel kernels") on a
 * device uint8 mask: fills mesh (vertices, triangles, MeshVolume,
 * SurfaceArea, voxel count).  Synchronises `stream` (the vertex and triangle
 * counts are returned in *mesh).  mask_dev: device, nx*ny*nz bytes, not
 * modified. */
rad_status rad_mesh(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], rad_mesh_t* mesh,
                    void* stream);

/* Marching cubes on a device float32 probability map (iso level 0.5,
 * linearly interpolated vertices); vtx_t is filled. */
rad_status rad_soft_mesh(const float* prob_dev, const int64_t dims[3], const double spacing[3], rad_mesh_t* mesh,
                         void* stream);

/* Diameters of a mesh (Sec. 2, "Parallel diameter calculation"): FP32
 * filter over tiled, bounding-box-culled vertex pairs, then FP64
 * confirmation of every pair within the filter's error bound, so the result
 * equals the FP64 all-pairs maximum.  Writes all features of the mesh to
 * *out (host).  Synchronises `stream`. */
rad_status rad_shape(const rad_mesh_t* mesh, rad_features_t* out, void* stream);

/* The same diameters by a plain FP64 all-pairs kernel (one thread block per
 * strip of pairs, no culling, no FP32 filter): the comparison kernel.
 * Writes all features of the mesh to *out.  Synchronises `stream`. */
rad_status rad_shape_plain_fp64(const rad_mesh_t* mesh, rad_features_t* out, void* stream);

/* Accumulation patterns of the FP64 diameter search (Sec. 3, "Optimization
 * research and results", optimisation steps (1)-(5), Fig. 3), plus the
 * culled search of rad_shape with FP64 in place of the FP32 filter:
 *   RAD_FP64_EQUAL_LOAD     (1) equal runs of pairs per thread, vertices read
 *                               from global memory, every improvement pushed
 *                               to the global result by an atomic;
 *   RAD_FP64_BLOCK_ATOMICS  (2) as (1), improvements kept per block in shared
 *                               memory, one global atomic per block;
 *   RAD_FP64_SHARED_2D      (3) tile pairs per block, the partner tile staged
 *                               in shared memory as a [vertex][xyz] array,
 *                               block result in shared memory as in (2);
 *   RAD_FP64_THREAD_LOCAL   (4) as (3) with per-thread maxima in registers,
 *                               merged once per block;
 *   RAD_FP64_PLAIN_1D       (5) per-coordinate 1D shared arrays, per-thread
 *                               maxima, one partial per block and a final
 *                               pass: the kernel of rad_shape_plain_fp64;
 *   RAD_FP64_CULLED             the tile walk and bounding-box culling of
 *                               rad_shape, every surviving pair evaluated in
 *                               FP64 (no FP32 filter, no candidate list).
 * Every variant returns the exact FP64 maxima with the smallest (i, j) on
 * ties, identical to rad_shape.  Any other value gives RAD_ERR_INVALID_ARG. */
enum {
  RAD_FP64_EQUAL_LOAD = 1,
  RAD_FP64_BLOCK_ATOMICS = 2,
  RAD_FP64_SHARED_2D = 3,
  RAD_FP64_THREAD_LOCAL = 4,
  RAD_FP64_PLAIN_1D = 5,
  RAD_FP64_CULLED = 6
};

/* Diameters of `mesh` by one of the variants above; all features of the
 * mesh to *out (host).  Synchronises `stream`. */
rad_status rad_shape_fp64_variant(const rad_mesh_t* mesh, int variant, rad_features_t* out, void* stream);

/* Whole path for one device mask: mesh + shape with library-owned buffers
 * kept in `ws` between calls (one host synchronisation per call, none
 * inside).  From the second call with the same (mask_dev, dims, spacing) and
 * unchanged pool sizes the whole pass is replayed as one captured CUDA graph.
 * *ws must be NULL on the first call; free with rad_workspace_free(). */
typedef struct rad_workspace rad_workspace_t;
rad_status rad_extract(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], rad_features_t* out,
                       rad_workspace_t** ws, void* stream);

/* Whole path for one HOST mask; the features are copied back.  A pinned
 * (page-locked, device-mapped) mask is read in place by the first kernel
 * over the host link, with no staging copy; the graph is replayed while the
 * mask's address stays the same.  A pageable mask is copied to a device
 * buffer inside the call first.  Either way the mask has been read when the
 * call returns.  Same workspace rules as rad_extract. */
rad_status rad_extract_host(const uint8_t* mask_host, const int64_t dims[3], const double spacing[3],
                            rad_features_t* out, rad_workspace_t** ws, void* stream);

void rad_workspace_free(rad_workspace_t* ws);
void rad_mesh_free(rad_mesh_t* mesh);

/* ---- batches of regions of interest ------------------------------------------ */

/* A batch of n_rois device uint8 masks of any sizes and spacings (ROI i:
 * masks_dev[i], dims[3 i .. 3 i + 2], spacing[3 i .. 3 i + 2]) processed
 * together: every stage of the mesh and of the diameters is one launch over
 * all ROIs (rows, vertices, tiles and tile pairs of every ROI share one
 * device work space), and the whole pass is captured once as a CUDA graph.
 * rad_batch_create validates the ROIs, sizes the pools with one counting
 * pass and runs + captures the pass (synchronises `stream`).  The masks are
 * read at every rad_batch_run (their contents may change; their addresses
 * and sizes may not).  Pool overflows after content changes are detected and
 * the pass re-runs with grown pools. */
typedef struct rad_batch rad_batch_t;
rad_status rad_batch_create(int n_rois, const uint8_t* const* masks_dev, const int64_t* dims, const double* spacing,
                            rad_batch_t** out, void* stream);

/* Replay the batch: out (host, n_rois entries) receives every ROI's
 * features.  Synchronises `stream`. */
rad_status rad_batch_run(rad_batch_t* batch, rad_features_t* out, void* stream);
void rad_batch_destroy(rad_batch_t* batch);

/* Copy a mesh's arrays to caller buffers (host or device; any may be NULL):
 * idx2 n_vertices x 3 int16, t n_vertices doubles (soft meshes only), tri
 * n_triangles x 3 int32.  Synchronises `stream`. */
rad_status rad_mesh_copy(const rad_mesh_t* mesh, int16_t* idx2, double* t, int32_t* tri, void* stream);

/* ---- soft probability maps: forward and adjoint ------------------------------ */

/* Forward pass on a device float32 probability map [nz][ny][nx] (iso level
 * 0.5, linearly interpolated vertices; a 0/1 map gives the mask's mesh):
 * out[0] = SurfaceArea, out[1] = MeshVolume, out[2] = Maximum3DDiameter
 * (host doubles); argmax = the diameter's vertex pair (host).  Uses and
 * keeps the buffers of *ws (NULL on first use).  Synchronises `stream`. */
rad_status rad_soft_forward(const float* prob_dev, const int64_t dims[3], const double spacing[3], double out[3],
                            int32_t argmax[2], rad_workspace_t** ws, void* stream);

/* Adjoint: grad_dev (device, nx*ny*nz doubles, overwritten) receives the
 * gradient of gout[0]*SurfaceArea + gout[1]*MeshVolume +
 * gout[2]*Maximum3DDiameter with respect to every voxel value.  The mesh is
 * recomputed from prob_dev (nothing of the forward pass is stored but the
 * argmax pair it returned, passed back here).  Mesh topology, triangulation
 * and the argmax pair are held fixed (the features are piecewise smooth).
 * Voxels away from the iso-surface get 0.  Synchronises `stream`. */
rad_status rad_soft_backward(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                             const double gout[3], const int32_t argmax[2], double* grad_dev, rad_workspace_t** ws,
                             void* stream);

/* All features of a soft map in *out (host), as rad_shape gives them for
 * its mesh: SurfaceArea, MeshVolume, VoxelVolume (voxels above 0.5), the
 * maximum 3D diameter and the planar diameters with their argmax pairs, and
 * the derived Shape features.  A plane of a soft mesh is the set of vertices
 * whose coordinate on that axis is exactly the same FP64 value (on a grid
 * plane, or off it where interpolated vertices of several edges coincide).
 * Synchronises `stream`. */
rad_status rad_soft_features(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                             rad_features_t* out, rad_workspace_t** ws, void* stream);

/* Adjoint with the planar diameters: grad_dev (device, nx*ny*nz doubles,
 * overwritten) receives the gradient of
 *   gout[0] A + gout[1] V + gout[2] D3 + gout[3] DSlice + gout[4] DColumn + gout[5] DRow
 * with the argmax pairs (argmax[2q], argmax[2q+1]) of the 3D, Slice, Column
 * and Row diameters from rad_soft_features (-1, -1 leaves a term out).  Each
 * pair is held fixed, a planar pair with its plane; otherwise as
 * rad_soft_backward.  Synchronises `stream`. */
rad_status rad_soft_backward_planes(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                                    const double gout[6], const int32_t argmax[8], double* grad_dev,
                                    rad_workspace_t** ws, void* stream);

/* Batches of soft maps: n maps (device float32 maps probs_dev[i] of size
 * dims[3i..3i+2] with spacing spacing[3i..3i+2]) through one set of launches
 * for the meshes, one for the diameters and one for the adjoint.
 * rad_soft_batch_forward writes out[0..n-1] (host) like rad_soft_features;
 * rad_soft_batch_backward writes each grads_dev[i] (device, overwritten) like
 * rad_soft_backward_planes, with weights gout[6i..6i+5] and argmax pairs
 * argmax[8i..8i+7].  n >= 1; any NULL pointer, bad size or spacing, or argmax
 * pair outside its map's mesh gives RAD_ERR_INVALID_ARG before any launch.
 * Synchronise `stream`. */
rad_status rad_soft_batch_forward(int n, const float* const* probs_dev, const int64_t* dims, const double* spacing,
                                  rad_features_t* out, rad_workspace_t** ws, void* stream);
rad_status rad_soft_batch_backward(int n, const float* const* probs_dev, const int64_t* dims, const double* spacing,
                                   const double* gout, const int32_t* argmax, double* const* grads_dev,
                                   rad_workspace_t** ws, void* stream);

/* ---- preprocessing: crop to the ROI and resample ------------------------------- */

/* Crop a device uint8 mask [nz][ny][nx] to the bounding box of its ROI
 * voxels and optionally resample it by nearest neighbour: the preprocessing
 * the paper names as open work that could move to the GPU (Sec. 3,
 * "Discussion of the results").  Definitions:
 *   ROI voxel   value == label (0 <= label <= 255), or value != 0 (label < 0);
 *   box         per axis the smallest and largest ROI index, widened by pad
 *               voxels per side and clamped to the grid: lo_k, m_k voxels;
 *   resample    (new_spacing non-NULL, every entry > 0) n'_k =
 *               floor((m_k - 1) s_k / s'_k) + 1 output voxels, output voxel i
 *               taking input voxel lo_k + min(m_k - 1, floor(i s'_k / s_k + 1/2))
 *               (FP64, left to right); without it the box itself (n'_k = m_k);
 *   output      1 where the sampled voxel is an ROI voxel, else 0.
 * Writes out_dims (n'_x, n'_y, n'_z), box_lo (the input index of output
 * voxel 0) and out_spacing (host) always; writes the output voxels to out_dev
 * (device, [n'_z][n'_y][n'_x] uint8, caller-owned) when out_capacity bytes
 * suffice, else returns RAD_ERR_CAPACITY having written nothing there (call
 * with out_capacity 0 to ask for the size).  A mask without ROI voxels gives
 * out_dims (0, 0, 0) and RAD_OK.  Scratch lives in *ws (NULL on first use).
 * Synchronises `stream`. */
rad_status rad_crop_resample(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], int label,
                             int pad, const double new_spacing[3], uint8_t* out_dev, int64_t out_capacity,
                             int64_t out_dims[3], int64_t box_lo[3], double out_spacing[3], rad_workspace_t** ws,
                             void* stream);

/* ---- measured arithmetic peaks -------------------------------------------- */

/* Kinds of rad_peak_probe. */
enum { RAD_PROBE_FP32 = 0, RAD_PROBE_FP32X2 = 1, RAD_PROBE_FP64 = 2 };

/* The arithmetic rate of this GPU, for the roofline of ALU-bound kernels
 * (the FP32 filter of the diameters, Sec. 2, is bound by FP32 arithmetic; the
 * plain all-pairs kernels by FP64).  One full wave of blocks runs eight
 * independent multiply-add chains per thread in registers, with no memory
 * traffic; the second of two identical launches is timed with CUDA events
 * on `stream` (a few ms each for FP32, about 10 ms for FP64).
 *   kind    RAD_PROBE_FP32 (scalar FP32 fma), RAD_PROBE_FP32X2 (packed f32x2
 *           fma, two lanes per instruction) or RAD_PROBE_FP64 (FP64 fma)
 *   tflops  host pointer; receives the rate in TFLOP/s, 2 flops per
 *           multiply-add (4 per packed one)
 * Unknown kind or NULL tflops: RAD_ERR_INVALID_ARG, nothing launched.  Uses a
 * 16-byte device buffer of its own (allocated and freed by the call).
 * Synchronises `stream`. */
rad_status rad_peak_probe(int kind, double* tflops, void* stream);

/* ---- failure detection check -------------------------------------------- */

/* Every device-side wait of the library (the look-back of its single-pass
 * scans) is bounded: after about 2^20 polls it gives up, sets a status bit
 * and the kernel returns, so a stuck wait becomes RAD_ERR_TIMEOUT on the host
 * instead of a hung GPU.  This call exercises that path on purpose: one warp
 * waits for a scan chunk that nothing ever publishes.  It returns
 * RAD_ERR_TIMEOUT (the expected outcome, after well under a second) with the
 * CUDA context still usable, or RAD_ERR_INTERNAL if the wait did not report.
 * Synchronises `stream`. */
rad_status rad_check_bounded_wait(void* stream);

/* ---- diameters without device allocation --------------------------------- */

/* The paper has no counterpart of this entry point; it exists for callers
 * that cannot call cudaMalloc (device memory owned by a framework's fixed
 * pool, services that forbid allocation after start-up, code that must avoid
 * the implicit synchronisation of cudaMalloc/cudaFree).  It computes the
 * same diameters as rad_shape_plain_fp64 (plain FP64 all pairs, same pinned
 * formula and tie-break) and allocates nothing: its only scratch is a static
 * device array of 256 KB built into the library, resident on a device from
 * the library module's load there until that device's context is destroyed.
 *   idx2_dev   device, n_vertices x 3 int16 doubled index coordinates
 *   t_dev      device, n_vertices doubles (soft meshes) or NULL (masks)
 *   n_vertices 0 .. 1048576 (4096 tiles of 256 vertices); larger counts are
 *              rejected with RAD_ERR_INVALID_ARG before any launch
 *   d2_dev     device, 4 doubles out: squared 3D, Slice, Column, Row diameter
 *   pairs_dev  device, 8 int32 out: (i, j) of each, (-1, -1) if no pair
 * Asynchronous on `stream` (nothing is copied to the host).  The first call
 * on a device looks up the device address of the static array with that
 * device current and caches it for the process: a device reset
 * (cudaDeviceReset) or another teardown of the device's primary context
 * invalidates that address, so no call may follow one.  All calls share the
 * one array: calls that overlap on the GPU (other streams or threads) race
 * and must be serialised by the caller. */
rad_status rad_diameters_plain_fp64_noalloc(const int16_t* idx2_dev, const double* t_dev, int64_t n_vertices,
                                            const double spacing[3], double* d2_dev, int32_t* pairs_dev,
                                            void* stream);

/* ---- configuration and introspection ----------------------------------- */

/* Set (non-NULL) and/or read (get non-NULL) the diameter tuning of the
 * calling process.  Invalid values return RAD_ERR_INVALID_ARG. */
rad_status rad_set_tuning(const rad_tuning_t* set, rad_tuning_t* get);

/* Per-kernel timing: when enabled, every kernel the library launches is
 * bracketed by CUDA events on its launch stream (inside a replayed graph the
 * event pairs are graph nodes, read after each replay).  rad_profile_read copies up
 * to `cap` records (name, launches, total milliseconds) and returns how many
 * exist; it synchronises the device.  rad_profile_reset clears them. */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
} rad_kernel_stat_t;
rad_status rad_profile_enable(int on);
int rad_profile_read(rad_kernel_stat_t* out, int cap);
void rad_profile_reset(void);

/* Number of kernels this library has launched in this process. */
int64_t rad_launch_count(void);

/* Statistics of the calling thread's last rad_shape / rad_extract /
 * rad_extract_host call (host copies; no device access). */
typedef struct {
  int64_t h2d_bytes, d2h_bytes;    /* host<->device bytes copied by the call */
  int64_t problems;                /* diameter problems: 1 (3D) + planes with >= 2 vertices */
  int64_t tiles, tile_pairs;       /* vertex tiles; tile pairs before culling */
  int64_t work_items;              /* tile pairs that survived the first culling pass */
  int64_t items_evaluated;         /* tile pairs evaluated in FP32 (after re-culling) */
  int64_t pairs_evaluated;         /* vertex pairs evaluated in FP32 */
  int64_t candidates;              /* pairs re-evaluated in FP64 */
  int64_t coarse_pairs;            /* coarse tile pairs refined (problems of 512+ tiles are walked at two levels) */
} rad_call_stats_t;
rad_status rad_last_call_stats(rad_call_stats_t* out);

const char* rad_status_str(rad_status s);
const char* rad_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H_ */
