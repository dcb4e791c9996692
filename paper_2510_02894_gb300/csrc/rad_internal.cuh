// Internal declarations shared by the CUDA translation units of librad.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>
#include <stdint.h>
#include <stdlib.h>

#include <string>
#include <vector>

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

// Kernels after the first of a pass are launched with programmatic stream
// serialization (unless per-kernel events are on): their CTAs are scheduled
// while the previous kernel drains and wait in pdl_enter() until it has
// completed and its writes are visible, which hides the launch gap between
// dependent kernels (also inside captured graphs).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

#define RAD_LAUNCH(name, kernel, grid, block, smem, stream, ...)                                   \
  do {                                                                                             \
    void* _tok = nullptr;                                                                          \
    ::rad::launch_begin(name, stream, &_tok);                                                      \
    cudaError_t _le = ::rad::launch_kernel(kernel, dim3(grid), dim3(block), (size_t)(smem), (stream), \
                                           _tok == nullptr, __VA_ARGS__);                          \
    if (_le == cudaSuccess) _le = cudaGetLastError();                                              \
    ::rad::launch_end(_tok, stream);                                                               \
    if (_le != cudaSuccess) return ::rad::cuda_fail(_le, name, __FILE__, __LINE__);                \
  } while (0)

// ---- single-pass scans (decoupled look-back) ------------------------------------
// Chunk c of a scan publishes its aggregate (flag 1) as soon as it has it and
// its inclusive prefix (flag 2) once it has looked back over its predecessors.
// Each quantity is one 64-bit word, flag << 62 | value, written and read whole,
// so no fence is needed between a value and its flag.  Chunks take their index
// from a ticket, so every chunk a block waits for is already running and
// publishes without waiting itself; only aggregates are waited for.  Every
// wait is bounded: after kScanSpinLimit polls the chunk is counted as zero and
// DEV_ERR_TIMEOUT is raised (the result is then reported as an error by the
// host, never used).
template <int Q>
struct __align__(16) ScanTile {
  unsigned long long w[Q];
};

constexpr unsigned int kScanSpinLimit = 1u << 20;
constexpr unsigned long long kScanValue = (1ull << 62) - 1ull;

// One thread: publish values (flag 1: aggregate, flag 2: inclusive prefix).
template <int Q>
__device__ __forceinline__ void scan_publish(ScanTile<Q>* t, const long long* v, unsigned long long flag) {
  for (int q = 0; q < Q; ++q)
    *(volatile unsigned long long*)&t->w[q] = (flag << 62) | ((unsigned long long)v[q] & kScanValue);
}

// One full warp: the exclusive prefix of chunk c > 0 (the same in every lane).
template <int Q>
__device__ void scan_lookback(ScanTile<Q>* tiles, int c, long long* excl, unsigned int* status) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < Q; ++q) {
    excl[q] = 0;
    for (int p = c - 1; p >= 0; p -= 32) {
      const int k = p - lane;  // lane l looks at chunk p - l
      unsigned long long x = 0;
      if (k >= 0) {
        x = *(volatile unsigned long long*)&tiles[k].w[q];
        for (unsigned int n = 0; (x >> 62) == 0 && n < kScanSpinLimit; ++n) {
          __nanosleep(32);
          x = *(volatile unsigned long long*)&tiles[k].w[q];
        }
        if ((x >> 62) == 0) atomicOr(status, 1u << 4);  // DEV_ERR_TIMEOUT
      }
      // the nearest predecessor with an inclusive prefix ends the look-back
      const unsigned int incl = __ballot_sync(0xffffffffu, k >= 0 && (x >> 62) == 2);
      const int stop = incl ? __ffs(incl) - 1 : 31;
      long long v = (k >= 0 && lane <= stop) ? (long long)(x & kScanValue) : 0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      excl[q] += v;
      if (incl) break;  // chunk 0 publishes its inclusive prefix at once, so this always ends
    }
  }
}

// Byte ranges that the first kernel of a stage zeroes (instead of memset
// nodes between kernels): 8-byte aligned, lengths rounded up to whole words
// inside their allocations.
struct ZeroSet {
  static constexpr int kMax = 8;
  unsigned long long* p[kMax];
  long long words[kMax];
  int count;
};

inline void zero_add(ZeroSet& z, void* p, size_t bytes) {
  if (z.count >= ZeroSet::kMax) abort();  // a fixed list: more ranges is a bug of the caller
  z.p[z.count] = static_cast<unsigned long long*>(p);
  z.words[z.count] = (long long)((bytes + 7) / 8);
  ++z.count;
}

__device__ __forceinline__ void zero_ranges(const ZeroSet& z) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (int k = 0; k < z.count; ++k)
    for (long long i = tid; i < z.words[k]; i += nth) z.p[k][i] = 0ull;
}

// First statement of every kernel: wait for the previous kernel in the stream
// (a no-op without a programmatic dependency), then let the next one be
// scheduled.  No kernel parameter of this library is declared restrict:
// with restrict-qualified parameters the compiler may treat loads of data
// that an earlier kernel of the pass writes as invariant (read-only cache
// loads, free to move above griddepcontrol.wait), and under programmatic
// dependent launch such loads were measured to return data from before the
// earlier kernel's writes.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

int num_sms();
bool profiling_on();
// CTAs of a kernel that are resident on one SM at once (cached per kernel,
// block size and device; at least 1).
int resident_ctas(const void* kernel, int threads, size_t smem);
// One full wave of a persistent (grid-stride) kernel, at most `needed` CTAs.
template <typename K>
int wave_grid(K kernel, int threads, long long needed, size_t smem = 0) {
  const long long wave = (long long)num_sms() * resident_ctas((const void*)kernel, threads, smem);
  return (int)std::max<long long>(1, std::min<long long>(needed, wave));
}
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
  DEV_ERR_PAIR = 1u << 7,     // an argmax pair passed to the soft adjoint is not a vertex pair of its mesh
};
static_assert(DEV_ERR_TIMEOUT == (1u << 4), "scan_lookback raises this bit");

// ---- marching cubes -----------------------------------------------------------
// One region of interest of a batch (host-computed, uploaded as a table).
struct Roi {
  const void* data;       // device mask (uint8) or probability map (float32)
  int nx, ny, nz, W;      // W: 32-bit words per bitset row
  int BY, BZ;             // bitset rows per axis: ny + 3, nz + 3 (zero padding)
  int vec16, tab;         // 16-byte loads possible; index of its case table
  long long R;            // owner / cube rows: (ny + 1) (nz + 1)
  long long row0, word0;  // first row and first bitset word in the batch
  long long wpre0;        // first per-word prefix slot
  double sx, sy, sz;
};

// Per-ROI results of a pass (device).
struct RoiOut {
  long long v0, nv, t0, nt, c0, na, nvox;  // id ranges of vertices, triangles, cubes; inside voxels
  long long vsum;                          // exact sum of A.(B x C) in half-voxel units (masks)
  double vol6, area2;                      // 6 V and 2 A
  // exact moments of the inside voxels' index coordinates:
  // sum x, y, z, xx, yy, zz, xy, xz, yz
  unsigned long long mom[9];
  // derived Shape features (rad_features_t order, Sphericity .. Flatness),
  // valid when has_derived (masks: computed beside the diameter stage)
  double derived[10];
  long long has_derived;
};


struct MeshTotals {  // batch-wide counts and status of one marching-cubes pass
  long long nv, nt, nvox, na;
  long long nwords;        // words with surface (binary masks: the emit kernel's work list)
  unsigned long long emit_ticket;  // next chunk of the word list
  unsigned int status;
  unsigned int done_ctas;  // last-CTA ticket of the soft cube kernel
  unsigned int mom_done;   // last-CTA ticket of the moments kernel
  unsigned int pad;
};

// Host view of a batch.
struct MeshBatch {
  int n = 0;
  bool soft = false;
  const Roi* rois = nullptr;  // device table
  long long rows = 0, words = 0, wpre = 0;
  int L = 1, Wc = 1;          // lanes per row group; word-loop bound
};

// Scratch of the marching-cubes pass, reused between calls.
struct MeshScratch {
  DevBuf bits;    // packed inside bits of every ROI
  DevBuf counts;  // int4 per row: vertices, triangles, inside voxels, active cubes
  DevBuf wpre;    // int per (row, word): row-local vertex prefix
  DevBuf tpre;    // int per (row, word): row-local triangle prefix
  DevBuf wlist;   // int2 per word with surface: (global row, word)
  DevBuf prefix;  // int64 x 4 per row: chunk-local exclusive prefixes
  DevBuf chunk;   // int64 x 4 per scan chunk: chunk offsets
  DevBuf cubes;   // int4 per active cube: x, global row, case, first triangle id
  DevBuf hist;    // uint64 x 256 per ROI: active cubes per case (mask area)
  DevBuf partial; // per-CTA FP64 partial sums of 6V and 2A (soft maps)
  DevBuf bintab;  // case tables, one per spacing
  DevBuf tabsp;   // spacings of the case tables
};

void plan_batch(const int64_t* dims, const void* const* data, const int* tab, const double* spacing, int n, bool soft,
                std::vector<Roi>& rois, MeshBatch& b);
// Case tables of binary masks, one per spacing (n_tabs x 3 doubles, host).
rad_status mesh_tables(const double* spacings_host, int n_tabs, MeshScratch& s, cudaStream_t st);
// Phase 1: pack + count + scan; batch totals in *tot, per-ROI id ranges in out[].
rad_status mesh_count(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, cudaStream_t st);
// Phase 2: vertices / triangles (up to the capacities) and per-ROI 6V, 2A.
// With totals = false a mask's per-ROI 6V and 2A are left to mesh_totals
// (on any stream ordered after this one).
rad_status mesh_emit(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, int16_t* idx2, double* vt,
                     int32_t* tri, long long vcap, long long tcap, cudaStream_t st, bool totals = true);
rad_status mesh_totals(const MeshBatch& b, MeshScratch& s, RoiOut* out, cudaStream_t st);
// Exact coordinate moments of every ROI's inside voxels from the packed bits,
// and from them the principal axes (after mesh_count; on any stream ordered
// after it).
rad_status mesh_moments(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, cudaStream_t st);

// ---- diameters ----------------------------------------------------------------
struct DiamScratch {
  DevBuf misc;        // sort, problems, tiles, work list, candidates (carved per run)
  DevBuf plain_part;  // per-CTA partial results of the plain FP64 kernel
  long long work_cap = 0, cand_cap = 0;
  bool fp64_pairs = false;  // evaluate the surviving tile pairs in FP64 (no FP32 filter)
};

// Per-ROI parameters of the diameter problems (host-computed, uploaded).
struct RoiDiam {
  int nx, ny, nz, planes;         // planes: also the planar diameters (masks)
  int cell_shift, CX, CY, CZ;     // 3D cells
  int plane_shift, PX, PY, PZ;    // in-plane 2D cells
  long long key0;                 // first sort key of the ROI
  long long C3, S0, S1, S2, K;    // key blocks (relative): 3D cells, Slice, Column, Row; total
  long long plane0;               // first plane of the ROI in the batch
  long long tab0;                 // masks: first entry of the ROI's FP32 coordinate tables; -1: none
  double sx, sy, sz;
  double cx, cy, cz;              // centre (index units)
  double alpha, beta, gamma;      // FP32 error-bound coefficients
};

// Per-ROI result (device): FP64 bits of the squared diameters and the
// (i << 32 | j) argmax pairs (ROI-local ids) for 3D, Slice, Column, Row.
struct DiamOut {
  unsigned long long d2[4];
  unsigned long long pair[4];
};

struct DiamStats {
  long long problems, tiles, tile_pairs, work_items, items_evaluated, pairs_evaluated, candidates;
  unsigned int status, coarse_pairs;
};

// Result of the plain FP64 kernel (one mask).
struct DiamResult {
  double d2[4];
  int i[4], j[4];
};

struct MeshDims {  // size of one grid
  int nx, ny, nz;
};
inline MeshDims make_dims(const int64_t dims[3]) { return MeshDims{(int)dims[0], (int)dims[1], (int)dims[2]}; }

void plan_diam(const std::vector<Roi>& rois, bool soft, std::vector<RoiDiam>& rd, long long& nkeys, long long& ntab,
               long long& nplanes);
// which: 1 = the stage's initialisation only (zeroing, per-ROI results,
// coordinate tables; needs nothing from the mesh), 2 = everything after it,
// 3 = both.  Both calls of a split run see the same scratch layout.
rad_status diam_run(int n, const RoiDiam* rd, const RoiOut* ro, const long long* nv_dev, long long nv_cap,
                    long long nkeys, long long nplanes, long long ntab, bool planes, const int16_t* idx2,
                    const double* vt, DiamScratch& s, DiamOut* out, DiamStats* stats, cudaStream_t st,
                    int which = 3);
rad_status diam_plain_fp64(const int16_t* idx2, const double* vt, long long nv, const MeshDims& d, const double sp[3],
                           DiamScratch& s, DiamResult* out_dev, cudaStream_t st);
// FP64 all-pairs diameters by one of the accumulation variants
// RAD_FP64_EQUAL_LOAD .. RAD_FP64_PLAIN_1D (one mesh; results as diam_plain_fp64).
rad_status diam_fp64_variant(int variant, const int16_t* idx2, const double* vt, long long nv, const MeshDims& d,
                             const double sp[3], DiamScratch& s, DiamResult* out_dev, cudaStream_t st);

const rad_tuning_t& tuning();

// Adjoint of the soft-map features (grad: dense FP64, nx*ny*nz; gvtx: 3 x vcap).
// One map of a soft adjoint batch (device table): its map and gradient
// (dense [nz][ny][nx] float64, caller-owned), size, spacing, the weights
// (A, V, D3, Slice, Column, Row) and the four argmax pairs (ROI-local vertex
// ids, -1: term left out), and its first voxel in the batch's voxel count.
struct SoftMap {
  const float* prob;
  double* grad;
  int nx, ny, nz, pad;
  double sx, sy, sz;
  double gout[6];
  int pair[8];
  long long vox0;
};

// Preprocessing (prep.cu): the ROI's box, widened and clamped (lo, m voxels
// per axis), and the output size; empty when the mask has no ROI voxel.
struct PrepInfo {
  long long lo[3], m[3], nout[3];
  int empty, pad;
};
// Box and output size of a crop/resample into *info_host (synchronises st).
rad_status prep_bbox(const uint8_t* mask, const int64_t dims[3], const double sp[3], int label, int pad,
                     const double* new_sp, DevBuf& scratch, PrepInfo* info_host, cudaStream_t st);
// The output voxels into out (info_host from prep_bbox on the same scratch; synchronises st).
rad_status prep_gather(const uint8_t* mask, const int64_t dims[3], const double sp[3], int label,
                       const double* new_sp, const PrepInfo& info_host, DevBuf& scratch, uint8_t* out,
                       cudaStream_t st);

// Gradients of a batch of soft maps whose meshes are in the pools (see soft.cu).
rad_status soft_adjoint(const int16_t* idx2, const double* vt, const int32_t* tri, const long long* nv_dev,
                        const long long* nt_dev, long long vcap, long long tcap, const RoiOut* ro, const SoftMap* maps,
                        int n, long long total_vox, double* gvtx, unsigned int* status, cudaStream_t st);

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

// A (d2, i, j) maximum as one 128-bit key: high word the bits of d2
// (non-negative doubles order like their bit patterns), low word
// ~(i << 32 | j), so the larger key has the larger d2, then the smaller
// (i, j).  Zero means "no pair yet".
struct __align__(16) Key128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ bool key_gt(const Key128& a, const Key128& b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

__device__ __forceinline__ Key128 make_key(double d2, int i, int j) {
  Key128 k;
  k.hi = (unsigned long long)__double_as_longlong(d2);
  k.lo = ~(((unsigned long long)(unsigned int)i << 32) | (unsigned int)j);
  return k;
}

// 128-bit compare-and-swap on a 16-byte aligned generic address (global or
// shared); returns the value found there.
__device__ __forceinline__ Key128 cas128(Key128* p, const Key128& cmp, const Key128& val) {
  Key128 r;
  asm volatile(
      "{\n\t.reg .b128 d, c, v;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.cas.b128 d, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(p)
      : "memory");
  return r;
}

// Raise *p to at least v; returns the larger of v and what *p held.  The
// first guess may be a torn read: the compare-and-swap validates it.
__device__ __forceinline__ Key128 atomic_max_key(Key128* p, const Key128& v) {
  Key128 cur;
  cur.lo = *(volatile unsigned long long*)&p->lo;
  cur.hi = *(volatile unsigned long long*)&p->hi;
  while (key_gt(v, cur)) {
    const Key128 prev = cas128(p, cur, v);
    if (prev.lo == cur.lo && prev.hi == cur.hi) return v;
    cur = prev;
  }
  return cur;
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
