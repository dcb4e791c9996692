// Internal declarations shared by the CUDA translation units of librad.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rad.h"

namespace rad {

// ---- error text ------------------------------------------------------------
void set_error(const char* fmt, ...);
rad_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define RAD_CUDA(call)                                                             \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) return ::rad::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define RAD_TRY(expr)                     \
  do {                                    \
    rad_status _s = (expr);               \
    if (_s != RAD_OK) return _s;          \
  } while (0)

// ---- kernel launch bookkeeping ---------------------------------------------
// Every kernel launch goes through RAD_LAUNCH: it counts the launch and, when
// profiling is on, brackets it with CUDA events on its own stream.
void launch_begin(const char* name, cudaStream_t s, void** token);
void launch_end(void* token, cudaStream_t s);

#define RAD_LAUNCH(name, kernel, grid, block, smem, stream, ...)     \
  do {                                                               \
    void* _tok = nullptr;                                            \
    ::rad::launch_begin(name, stream, &_tok);                        \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);      \
    cudaError_t _le = cudaGetLastError();                            \
    ::rad::launch_end(_tok, stream);                                 \
    if (_le != cudaSuccess) return ::rad::cuda_fail(_le, name, __FILE__, __LINE__); \
  } while (0)

int num_sms();
bool profiling_on();
long long alloc_epoch();           // bumps whenever a library buffer is reallocated

// ---- device buffers ----------------------------------------------------------
// A grow-only device buffer owned by the library.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  rad_status reserve(size_t need);
  void release();
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Device-side status word: kernels OR error bits into it; the host reads it
// at the end of a call.
enum : uint32_t {
  DEV_ERR_VCAP = 1u << 0,     // vertex pool too small
  DEV_ERR_TCAP = 1u << 1,     // triangle pool too small
  DEV_ERR_CANDCAP = 1u << 2,  // candidate pair pool too small
  DEV_ERR_WORKCAP = 1u << 3,  // tile-pair work list too small
  DEV_ERR_TIMEOUT = 1u << 4,  // a bounded wait gave up
  DEV_ERR_INTERNAL = 1u << 5, // consistency check failed
  DEV_ERR_PROBCAP = 1u << 6,  // problem/tile list too small
};

// ---- marching cubes -----------------------------------------------------------
struct MeshDims {
  int nx, ny, nz;
  int W;       // 32-bit words per bitset row
  int BY, BZ;  // bitset rows per axis (ny + 3, nz + 3)
  int64_t R;   // owner / cube rows: (ny + 1) * (nz + 1)
};
MeshDims make_dims(const int64_t dims[3]);

// Scratch of the marching-cubes pass, reused between calls.
struct MeshScratch {
  DevBuf bits;    // packed inside bits, (ny + 3) (nz + 3) rows of W words
  DevBuf counts;  // int4 per row: vertices, triangles, inside voxels, active cubes
  DevBuf wpre;    // int per (row, word): row-local vertex prefix
  DevBuf prefix;  // int64 x 3 per row: chunk-local exclusive prefixes (vertices, triangles, cubes)
  DevBuf chunk;   // int64 x 4 per scan chunk: chunk offsets (and inside voxels)
  DevBuf cubes;   // int4 per active cube: x, row, case, first triangle id
  DevBuf hist;    // uint64 x 256: active cubes per case (mask area)
  DevBuf partial; // per-CTA FP64 partial sums of 6V and 2A (soft maps)
  DevBuf bintab;  // per-spacing binary case table
  double tab_spacing[3] = {0, 0, 0};
  bool tab_valid = false;
};

struct MeshTotals {  // device counts and sums of one marching-cubes pass
  long long nv, nt, nvox, na;
  double vol6, area2;
  long long vsum;          // exact sum of A.(B x C) in half-voxel units (masks)
  unsigned int status;
  unsigned int done_ctas;  // last-CTA ticket of the cube kernel
};

// Phase 1: pack + count + scan; the counts land in *tot (device).
rad_status mesh_count(const void* data, bool soft, const MeshDims& d, MeshScratch& s, MeshTotals* tot,
                      cudaStream_t st);
// Phase 2: emit vertices / triangles (up to the given capacities) and reduce
// 6V and 2A into *tot.
rad_status mesh_emit(const void* data, bool soft, const MeshDims& d, const double sp[3], MeshScratch& s,
                     MeshTotals* tot, int16_t* idx2, double* vt, int32_t* tri, long long vcap, long long tcap,
                     cudaStream_t st);

// ---- diameters ----------------------------------------------------------------
struct DiamScratch {
  DevBuf misc;        // sort, problems, tiles, work list, candidates (carved per run)
  DevBuf plain_part;  // per-CTA partial results of the plain FP64 kernel
  long long work_cap = 0, cand_cap = 0;
};

// Device result of one diameter run: for 3D, Slice, Column, Row.
struct DiamResult {
  double d2[4];
  int i[4], j[4];
  long long problems, tiles, tile_pairs, work_items, items_evaluated, pairs_evaluated, candidates;
};

rad_status diam_run(const int16_t* idx2, const double* vt, long long nv_hint, const long long* nv_dev,
                    const MeshDims& d, const double sp[3], DiamScratch& s, DiamResult* out_dev,
                    unsigned int* status_dev, cudaStream_t st);
rad_status diam_plain_fp64(const int16_t* idx2, const double* vt, long long nv, const MeshDims& d, const double sp[3],
                           DiamScratch& s, DiamResult* out_dev, cudaStream_t st);

const rad_tuning_t& tuning();

// Adjoint of the soft-map features (grad: dense FP64, nx*ny*nz; gvtx: 3 x vcap).
rad_status soft_adjoint(const int16_t* idx2, const double* vt, const int32_t* tri, const long long* nv_dev,
                        const long long* nt_dev, long long vcap, long long tcap, const float* prob, const MeshDims& d,
                        const double sp[3], const double gout[3], int ai, int aj, double* gvtx, double* grad,
                        cudaStream_t st);

}  // namespace rad

// ---- pinned FP64 arithmetic (no contraction) ------------------------------------
__device__ __forceinline__ double pin_tri_r(const double* A, const double* B, const double* C) {
  double e1x = __dsub_rn(B[0], A[0]), e1y = __dsub_rn(B[1], A[1]), e1z = __dsub_rn(B[2], A[2]);
  double e2x = __dsub_rn(C[0], A[0]), e2y = __dsub_rn(C[1], A[1]), e2z = __dsub_rn(C[2], A[2]);
  double nx = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
  double ny = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
  double nz = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
  double s = __dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny));
  s = __dadd_rn(s, __dmul_rn(nz, nz));
  return __dsqrt_rn(s);
}

__device__ __forceinline__ double pin_vol6(const double* A, const double* B, const double* C) {
  double k0 = __dsub_rn(__dmul_rn(B[1], C[2]), __dmul_rn(B[2], C[1]));
  double k1 = __dsub_rn(__dmul_rn(B[2], C[0]), __dmul_rn(B[0], C[2]));
  double k2 = __dsub_rn(__dmul_rn(B[0], C[1]), __dmul_rn(B[1], C[0]));
  double r = __dmul_rn(A[0], k0);
  r = __dadd_rn(r, __dmul_rn(A[1], k1));
  r = __dadd_rn(r, __dmul_rn(A[2], k2));
  return r;
}

// Pinned squared distance of two index-space positions (FP64, left to right).
__device__ __forceinline__ double pin_d2(double uix, double uiy, double uiz, double ujx, double ujy, double ujz,
                                         double sx, double sy, double sz) {
  double dx = __dmul_rn(__dsub_rn(uix, ujx), sx);
  double dy = __dmul_rn(__dsub_rn(uiy, ujy), sy);
  double dz = __dmul_rn(__dsub_rn(uiz, ujz), sz);
  double r = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return __dadd_rn(r, __dmul_rn(dz, dz));
}

// Index-space position of a vertex from its doubled coordinates and t.
__device__ __forceinline__ void vertex_u(const int16_t* idx2, const double* vt, long long v, double u[3]) {
  int q0 = idx2[3 * v], q1 = idx2[3 * v + 1], q2 = idx2[3 * v + 2];
  if (vt == nullptr) {
    u[0] = 0.5 * (double)q0;
    u[1] = 0.5 * (double)q1;
    u[2] = 0.5 * (double)q2;
  } else {
    // the odd doubled coordinate marks the edge axis: u = g + t there
    double t = vt[v];
    u[0] = (q0 & 1) ? __dadd_rn((double)((q0 - 1) >> 1), t) : 0.5 * (double)q0;
    u[1] = (q1 & 1) ? __dadd_rn((double)((q1 - 1) >> 1), t) : 0.5 * (double)q1;
    u[2] = (q2 & 1) ? __dadd_rn((double)((q2 - 1) >> 1), t) : 0.5 * (double)q2;
  }
}
