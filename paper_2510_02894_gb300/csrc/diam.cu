// Maximum 3D and planar diameters over the mesh vertices (paper Sec. 2,
// "Parallel diameter calculation": each thread scans a subset of vertex pairs
// into a local maximum, then a reduction combines the local maxima).
//
// A batch of regions of interest (ROIs) runs as one set of launches: every
// problem carries its ROI, whose spacing, centre and error-bound coefficients
// live in a small device table.
//
// GB300 design (FP32 filter, FP64 confirmation):
//   1. Every vertex gets four keys -- a spatial cell (3D problem) and its
//      Slice (z), Column (y) and Row (x) plane -- and one counting sort lays
//      the vertices out as float4 (x, y, z in FP32, centred and scaled; w =
//      the FP32 squared norm), with the vertex ids in a parallel array.  A
//      mask's FP32 coordinates come from per-ROI tables indexed by the doubled
//      grid coordinate.  The 3D problem is the whole cell-sorted range; every
//      plane with two or more vertices is its own problem.
//   2. Each problem is cut into tiles of TS vertices with bounding boxes and
//      a representative vertex.  The upper triangle of a problem's tile pairs
//      is walked as (tile row, 128-column chunk) items spread evenly over all
//      warps: the representative pairs seed the running maximum F, then the
//      tile pairs whose farthest-corner bound reaches T(F) form the work list.
//   3. The surviving tile pairs are split into (tile pair, two 32-entry B
//      slices) warp units, dealt statically over all warps.  Every warp
//      evaluates its units in FP32 (f32x2, two A entries per lane and
//      coordinate) from its own shared-memory buffers (the next unit is
//      staged with cp.async while the current one is evaluated, no block
//      barriers); it re-culls against the current T before every slice,
//      keeps each slice maximum and raises F with one atomic when it beats F.
//      Slices whose maximum reaches the final T(F) are rescanned and their
//      pairs with f >= T(F) become candidates.
//   4. The candidates are re-evaluated in FP64 with the pinned formula: the
//      largest d2 per ROI and category, then the smallest (i, j) attaining it.
//
// FP32 error bounds (per pair, binary or soft; u = 2^-24, positions a relative
// to the grid centre, R = the grid's half diagonal in mm, d2 the FP64 value):
//   P = fl32(a), and once per entry n = fl(fl(P_x P_x + P_y P_y) + P_z P_z).
//   Pair kernels (expansion form, 3 FP32 operations per pair, n_i added once
//   per maximum):
//     h = fma(-2P_ix, P_jx, fma(-2P_iy, P_jy, fma(-2P_iz, P_jz, n_j)))
//     g = fl(n_i + h)
//     |g - d2| <= 4.1u R sqrt(d2) + 20.2u R^2
//     (the norms carry 2 gamma_3 R^2, the fma chain gamma_3 (|n_j| + 2 |P_i|
//     |P_j|) <= 3 gamma_3 R^2, the final add u |g| <= 4u R^2: about 19.1u R^2;
//     the FP32 positions 4u R sqrt(d2) + 4u^2 R^2)
//   Seed and box bounds (difference form):
//     dx = fl(P_i - P_j), f = fma(dz,dz, fma(dy,dy, dx*dx))
//     |f - d2| <= 5.1u d2 + 4.1u R sqrt(d2) + 4.1u^2 R^2.
// T(F) inverts the larger coefficient of each term (every coefficient
// doubled), so every pair attaining the FP64 maximum has g >= T(F) and
// f >= T(F) for any F not above the largest g or f of any pair; the culling
// bound uses the difference form's monotone FP32 operations on box distances,
// so it bounds f from above without any epsilon.  T only grows, so a pair
// culled or left out against an earlier T is also below the final one.
#include <atomic>
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "rad_internal.cuh"

namespace rad {

namespace {

constexpr int kChunk = 128;  // tile columns per seed / cull item (4 per lane)
// Problems of kBigTiles or more tiles are walked at two levels: coarse tiles
// of kCoarse tiles are seeded and culled first, then only the tile pairs
// inside surviving coarse pairs are tested (one warp per coarse pair).
constexpr int kCoarse = 32;
constexpr int kBigTiles = 512;

struct Problem {
  int axis;  // -1: 3D, 0: Row (equal x), 1: Column (equal y), 2: Slice (equal z)
  int beg, len;
  int tile_beg;  // first tile
  int roi;
  int q;   // result slot: 0 3D, 1 Slice, 2 Column, 3 Row
  int nt;  // tiles
  int fine;  // -1: walked as is; -2: tiles only (walked through its coarse problem, the next slot);
             // >= 0: coarse problem, first tile of its fine problem (the previous slot)
  long long chunk_end;  // one past the last seed/cull chunk of its rows; -1: past 2^31 chunks
};

struct __align__(16) Tile {
  int problem, beg, len, tile_end;  // tile_end: one past the problem's last tile
  int roi, q;                       // ROI and result slot of the problem
  int fine0, nfine;                 // coarse tiles: first fine tile and how many (else 0, 0)
};

// A surviving tile pair: both vertex ranges, its box bound and its result slot.
// A coarse tile pair that survived culling: its fine tile ranges.
struct RefineItem {
  int fa, na, fb, nb;
  int problem, roi, q, same;  // problem: the fine problem's slot; same: a coarse tile with itself
};

struct WorkItem {
  int problem, roi;
  int abeg, alen, bbeg, blen;
  float ub;
  int q;
};

struct Cand {
  int ea, eb, roi, q;  // sorted-entry indices of the pair, ROI, result slot
};

struct __align__(8) ProblemState {  // read as one 64-bit word by the pair kernel
  unsigned int F;  // float bits of the running FP32 maximum
  unsigned int T;  // float bits of T(F), raised with F
};

struct Counters {
  int n_problems;
  unsigned int alloc_fine;   // tiles of fine problems (their own region after the walked tiles)
  unsigned long long alloc;  // (seed/cull chunks << 32) + tiles, one atomic per problem
  long long n_pairs;         // tile pairs (upper triangles)
  long long n_work;
  long long n_cand;
  long long n_hits;  // slices to rescan for candidates
  unsigned long long items_evaluated, pairs_evaluated;
  unsigned int status;
  unsigned int n_refine;     // surviving coarse tile pairs
  unsigned int seed_done;  // last-block ticket of the seed
  unsigned int n_groups;   // planes of a soft map off the grid planes (groups of equal coordinate)
  unsigned int confirm_done, pad3;  // last-block ticket of the FP64 confirmation
};

// Batch-wide parameters of one run.
struct Params {
  int n;              // ROIs
  int TS;
  long long nplanes;  // planes of all ROIs
  long long work_cap, cand_cap, max_problems, max_tiles;
  long long max_fine, refine_cap;  // tiles of fine problems (their region after max_tiles); coarse pairs
  long long nv_cap;   // vertex pool capacity: device counts are clamped to it
  long long sweep_min;  // ROIs with at least this many vertices get the farthest-point seed
};

// Planes of soft maps.  A soft vertex lies on a grid edge: on the edge's
// axis its coordinate is g + t.  Where that value is an integer the vertex
// lies on a grid plane, and it joins that plane's problem like a mask vertex.
// Otherwise its plane (the vertices whose coordinate on that axis is exactly
// the same FP64 value, as the definition of the planar diameters asks) is
// found through a hash table keyed by (ROI, axis, value bits): every group of
// two or more vertices becomes one problem with a key of its own after all
// ROIs' keys; vertices alone on their value go to one spare key that no
// problem covers.
struct FracState {
  Key128* hkey = nullptr;  // (value bits, (ROI << 2 | axis) + 1); zero: empty slot
  int* hcnt = nullptr;     // vertices per slot
  int* hgid = nullptr;     // group of a slot with two or more vertices
  int* vslot = nullptr;    // slot of each vertex, -1: on a grid plane
  int* gra = nullptr;      // (ROI << 2 | axis) of each group
  long long hmask = 0;     // table size - 1 (a power of two at least twice the vertex capacity)
  long long fbase = 0;     // key of group 0
  long long gcap = 0;      // group keys (the spare key is fbase + gcap)
};

// Expansion form: a2 = (-2 P_i, n_i), b = (P_j, n_j).  The FMA chain starts
// from n_j and n_i is added last, so a maximum over many b needs that add
// only once (rounding to nearest is monotone: max fl(n_i + h) = fl(n_i + max h)).
__device__ __forceinline__ float pair_h(float4 a2, float4 b) {
  float h = __fmaf_rn(a2.z, b.z, b.w);
  h = __fmaf_rn(a2.y, b.y, h);
  return __fmaf_rn(a2.x, b.x, h);
}
__device__ __forceinline__ float pair_g(float4 a2, float4 b) { return __fadd_rn(a2.w, pair_h(a2, b)); }

// Packed pairs of FP32 values (Blackwell f32x2 arithmetic, round to nearest
// per element: the same results as the scalar operations).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpk2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float4 expand_a(float4 a) {
  return make_float4(__fmul_rn(-2.0f, a.x), __fmul_rn(-2.0f, a.y), __fmul_rn(-2.0f, a.z), a.w);
}

__device__ __forceinline__ float pair_f(float4 a, float4 b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  float f = __fmul_rn(dx, dx);
  f = __fmaf_rn(dy, dy, f);
  return __fmaf_rn(dz, dz, f);
}

// Threshold T(F): every pair attaining the FP64 maximum has f >= T(F).
__device__ __forceinline__ float threshold(float F, const RoiDiam& p) {
  const double f = (double)F;
  if (!(f > p.gamma)) return 0.0f;
  const double a1 = 1.0 + p.alpha;
  const double s = (-p.beta + sqrt(p.beta * p.beta + 4.0 * a1 * (f - p.gamma))) / (2.0 * a1);
  const double t = (1.0 - p.alpha) * s * s - p.beta * s - p.gamma;
  return t > 0.0 ? __double2float_rd(t) : 0.0f;
}

// Upper bound of f over all pairs of two boxes (same monotone operations).
__device__ __forceinline__ float box_ub(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  const float mx = fmaxf(__fsub_rn(bhi.x, alo.x), __fsub_rn(ahi.x, blo.x));
  const float my = fmaxf(__fsub_rn(bhi.y, alo.y), __fsub_rn(ahi.y, blo.y));
  const float mz = fmaxf(__fsub_rn(bhi.z, alo.z), __fsub_rn(ahi.z, blo.z));
  float f = __fmul_rn(mx, mx);
  f = __fmaf_rn(my, my, f);
  return __fmaf_rn(mz, mz, f);
}

__device__ __forceinline__ void vertex_q(const int16_t* idx2, long long v, int q[3]) {
  q[0] = idx2[3 * v];
  q[1] = idx2[3 * v + 1];
  q[2] = idx2[3 * v + 2];
}

__device__ __forceinline__ int slot_of_axis(int axis) { return axis < 0 ? 0 : (axis == 2 ? 1 : (axis == 1 ? 2 : 3)); }

// Running maximum F and threshold T are shared by a family: (ROI, result
// slot).  A family's result is the maximum over all of its problems (the 3D
// problem, or every plane of one orientation), so a tile pair of one plane
// whose bound is below the largest value found in ANY plane of its family
// cannot change the result and is culled.
__device__ __forceinline__ int fam_of(int roi, int q) { return 4 * roi + q; }

// ---- 1. keys, histogram, scatter ------------------------------------------------
// kind 0: 3D cell (z, y, x order); kinds 1..3: (plane, 2D cell) for Slice
// (equal z), Column (equal y) and Row (equal x), all offset by the ROI's
// first key.  Sorting by these keys gives every 3D problem spatially compact
// tiles and every plane compact 2D tiles.

__device__ __forceinline__ long long key_of(const RoiDiam& p, const int q[3], int kind) {
  const int x1 = q[0] + 1, y1 = q[1] + 1, z1 = q[2] + 1;  // 0 .. 2n
  if (kind == 0) {
    const int cx = x1 >> p.cell_shift, cy = y1 >> p.cell_shift, cz = z1 >> p.cell_shift;
    return p.key0 + ((long long)cz * p.CY + cy) * p.CX + cx;
  }
  const int px = x1 >> p.plane_shift, py = y1 >> p.plane_shift, pz = z1 >> p.plane_shift;
  if (kind == 1) return p.key0 + p.S0 + (long long)z1 * p.PX * p.PY + (long long)py * p.PX + px;
  if (kind == 2) return p.key0 + p.S1 + (long long)y1 * p.PX * p.PZ + (long long)pz * p.PX + px;
  return p.key0 + p.S2 + (long long)x1 * p.PY * p.PZ + (long long)pz * p.PY + py;
}

// Plane key (kinds 1..3) of vertex v: a mask vertex, or a soft vertex off
// its edge's axis, by key_of; a soft vertex on a grid plane by key_of with
// its exact doubled coordinate; otherwise its group's key (see FracState).
__device__ __forceinline__ long long plane_key(const RoiDiam& r, const int q[3], int kind, long long v,
                                               const double* vt, const FracState& fs) {
  const int a = 3 - kind;  // Slice: z, Column: y, Row: x
  if (vt == nullptr || !(q[a] & 1)) return key_of(r, q, kind);
  const double u = __dadd_rn((double)((q[a] - 1) >> 1), vt[v]);
  if (u == floor(u)) {
    int qq[3] = {q[0], q[1], q[2]};
    qq[a] = 2 * (int)u;
    return key_of(r, qq, kind);
  }
  const int h = fs.vslot[v];
  if (h >= 0 && fs.hcnt[h] >= 2) return fs.fbase + fs.hgid[h];
  return fs.fbase + fs.gcap;
}

// ROI of a global vertex id (last ROI whose first vertex is <= v).
__device__ __forceinline__ int roi_of_vertex(const RoiOut* ro, int n, long long v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ro[mid].v0 <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// FP32 position of vertex v relative to its ROI's centre, scaled by the
// spacing: a mask's coordinates come from the ROI's tables (indexed by the
// doubled grid coordinate), a soft map's from its FP64 position.
__device__ __forceinline__ float3 vert_pos(const int16_t* idx2, const double* vt, const float* ctab, const RoiDiam& r,
                                           long long v) {
  if (vt == nullptr) {
    const float* tx = ctab + r.tab0;
    const float* ty = tx + 2 * r.nx + 3;
    const float* tz = ty + 2 * r.ny + 3;
    return make_float3(tx[idx2[3 * v] + 2], ty[idx2[3 * v + 1] + 2], tz[idx2[3 * v + 2] + 2]);
  }
  double u[3];
  vertex_u(idx2, vt, v, u);
  return make_float3(__double2float_rn((u[0] - r.cx) * r.sx), __double2float_rn((u[1] - r.cy) * r.sy),
                     __double2float_rn((u[2] - r.cz) * r.sz));
}

__device__ __forceinline__ float pair_f3(float3 a, float3 b) {
  return pair_f(make_float4(a.x, a.y, a.z, 0.f), make_float4(b.x, b.y, b.z, 0.f));
}

// Farthest-point sweep of the 3D seed, accumulated per thread: the largest
// (f bits << 32 | ROI-local vertex) of the thread's vertices, for its current
// ROI.  f is the distance of an actual vertex pair, so it is a valid seed of
// the ROI's 3D family F; the argmax is kept when a slot array is given.
struct SweepAcc {
  int roi = -1;
  unsigned long long key = 0ull;
};

__device__ __forceinline__ void sweep_global(int roi, unsigned long long key, unsigned long long* slot,
                                             ProblemState* ps) {
  if (roi < 0 || key == 0ull) return;
  if (slot) atomicMax(&slot[roi], key);
  atomicMax(&ps[fam_of(roi, 0)].F, (unsigned int)(key >> 32));
}

// One step, called by every lane of the warp.  A single mask accumulates in
// the thread (one ROI; the block reduces at the end); a batch reduces the
// lanes of each ROI in the warp at once and makes one atomic per ROI.
__device__ __forceinline__ void sweep_step(SweepAcc& a, bool multi, bool valid, int roi, float f, unsigned int local,
                                           unsigned long long* slot, ProblemState* ps) {
  const unsigned long long k = valid ? ((unsigned long long)__float_as_uint(f) << 32) | local : 0ull;  // f >= 0
  if (!multi) {
    a.roi = 0;
    a.key = k > a.key ? k : a.key;
    return;
  }
  const int lane = threadIdx.x & 31;
  const unsigned int peers = __match_any_sync(0xffffffffu, valid ? roi : -1);
  const unsigned int hi = __reduce_max_sync(peers, (unsigned int)(k >> 32));
  const unsigned int lo = __reduce_max_sync(peers, (unsigned int)(k >> 32) == hi ? (unsigned int)k : 0u);
  if (valid && lane == __ffs(peers) - 1) sweep_global(roi, ((unsigned long long)hi << 32) | lo, slot, ps);
}

// End of the kernel (every thread of the block): lanes of one ROI reduce in
// the warp; warps whose ROI is the block's (all of them for a single mask)
// reduce in shared memory, so a block makes one atomic per value.
__device__ __forceinline__ void sweep_finish(const SweepAcc& a, int block_roi, unsigned long long* s_key,
                                             unsigned long long* slot, ProblemState* ps) {
  if (a.roi < 0 && block_roi < 0) return;  // block-uniform: a batch, or a block without vertices
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) *s_key = 0ull;
  __syncthreads();
  const unsigned int peers = __match_any_sync(0xffffffffu, a.roi);
  const unsigned int hi = __reduce_max_sync(peers, (unsigned int)(a.key >> 32));
  const unsigned int lo = __reduce_max_sync(peers, (unsigned int)(a.key >> 32) == hi ? (unsigned int)a.key : 0u);
  const unsigned long long k = ((unsigned long long)hi << 32) | lo;
  if (lane == __ffs(peers) - 1 && a.roi >= 0) {
    if (a.roi == block_roi) atomicMax(s_key, k);
    else sweep_global(a.roi, k, slot, ps);
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_global(block_roi, *s_key, slot, ps);
}

// fmix64, the finalizer of MurmurHash3 (Appleby): a 64-bit mixing function.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// Soft maps: every vertex whose coordinate on its edge's axis is not an
// integer enters the hash table (open addressing, linear probing, slots
// claimed by a 128-bit compare-and-swap) and counts itself in its slot.
__global__ void k_frac_insert(const int16_t* idx2, const double* vt, const long long* nv_dev, const RoiOut* ro,
                              Params p, FracState fs, Counters* cnt) {
  pdl_enter();
  const long long n = min(*nv_dev, p.nv_cap);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    int q[3];
    vertex_q(idx2, v, q);
    const int a = (q[0] & 1) ? 0 : ((q[1] & 1) ? 1 : 2);
    const double u = __dadd_rn((double)((q[a] - 1) >> 1), vt[v]);
    int slot = -1;
    if (u != floor(u)) {
      const int roi = p.n == 1 ? 0 : roi_of_vertex(ro, p.n, v);
      Key128 key;
      key.lo = (unsigned long long)__double_as_longlong(u);
      key.hi = (((unsigned long long)roi << 2) | (unsigned long long)a) + 1ull;
      long long h = (long long)(mix64(key.lo ^ mix64(key.hi)) & (unsigned long long)fs.hmask);
      for (long long probe = 0; probe <= fs.hmask; ++probe) {
        const Key128 old = cas128(&fs.hkey[h], Key128{0ull, 0ull}, key);
        if ((old.lo == 0ull && old.hi == 0ull) || (old.lo == key.lo && old.hi == key.hi)) {
          slot = (int)h;
          break;
        }
        h = (h + 1) & fs.hmask;
      }
      if (slot >= 0) atomicAdd(&fs.hcnt[slot], 1);
      else atomicOr(&cnt->status, DEV_ERR_PROBCAP);  // a full table: not reached at twice the vertex capacity
    }
    fs.vslot[v] = slot;
  }
}

// Every slot with two or more vertices becomes a group (a planar problem).
__global__ void k_frac_assign(FracState fs, Counters* cnt) {
  pdl_enter();
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h <= fs.hmask;
       h += (long long)gridDim.x * blockDim.x) {
    if (fs.hcnt[h] < 2) continue;
    const unsigned int g = atomicAdd(&cnt->n_groups, 1u);
    if ((long long)g < fs.gcap) {
      fs.hgid[h] = (int)g;
      fs.gra[g] = (int)(fs.hkey[h].hi - 1ull);
    } else {
      fs.hgid[h] = (int)fs.gcap;  // the spare key; reported
      atomicOr(&cnt->status, DEV_ERR_PROBCAP);
    }
  }
}

// Key histogram, warp-aggregated: lanes with equal keys (consecutive vertices
// share cells and planes) make one atomic.  Also the first sweep of the 3D
// seed: the vertex farthest from each ROI's first vertex.
__global__ void k_hist(const int16_t* idx2, const double* vt,
                       const long long* nv_dev, const RoiDiam* rd,
                       const RoiOut* ro, Params p, const float* ctab,
                       int* hist, unsigned long long* sweep, ProblemState* ps, FracState fs) {
  pdl_enter();
  __shared__ unsigned long long s_key;
  const long long n = min(*nv_dev, p.nv_cap);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  SweepAcc acc;
  for (long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; v0 < n; v0 += stride) {
    const long long v = v0 + lane;
    int q[3] = {0, 0, 0};
    int roi = 0;
    float f = 0.0f;
    unsigned int local = 0;
    bool sw = false;
    if (v < n) {
      vertex_q(idx2, v, q);
      roi = p.n == 1 ? 0 : roi_of_vertex(ro, p.n, v);
      sw = ro[roi].nv >= p.sweep_min;
      if (sw) {
        const long long first = ro[roi].v0;
        f = pair_f3(vert_pos(idx2, vt, ctab, rd[roi], first), vert_pos(idx2, vt, ctab, rd[roi], v));
        local = (unsigned int)(v - first);
      }
    }
    if (__any_sync(0xffffffffu, sw)) sweep_step(acc, p.n > 1, sw, roi, f, local, sweep, ps);
    const RoiDiam& r = rd[roi];
    for (int k = 0; k < 4; ++k) {
      const bool use = v < n && (k == 0 || r.planes);
      const long long key = use ? (k == 0 ? key_of(r, q, 0) : plane_key(r, q, k, v, vt, fs)) : -1;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[key], __popc(peers));
    }
  }
  sweep_finish(acc, p.n == 1 && blockIdx.x * (long long)blockDim.x < n ? 0 : -1, &s_key, sweep, ps);
}


// The four slot reservations of a warp are issued back to back, so one
// round trip covers all of them.
// The second sweep of the 3D seed rides along: each vertex's f to the vertex
// the first sweep found raises the ROI's 3D F.
__global__ void k_scatter(const int16_t* idx2, const double* vt,
                          const long long* nv_dev, const RoiDiam* rd,
                          const RoiOut* ro, Params p, const long long* offs,
                          int* cursor, const float* ctab,
                          float4* sorted, int* ids,
                          const unsigned long long* sweep, ProblemState* ps, FracState fs) {
  pdl_enter();
  __shared__ unsigned long long s_key;
  SweepAcc acc;
  const long long n = min(*nv_dev, p.nv_cap);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; v0 < n; v0 += stride) {
    const long long v = v0 + lane;
    int q[3] = {0, 0, 0};
    int roi = 0;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    float f2 = 0.0f;
    bool sw = false;
    if (v < n) {
      vertex_q(idx2, v, q);
      roi = p.n == 1 ? 0 : roi_of_vertex(ro, p.n, v);
      const RoiDiam& r = rd[roi];
      const float3 P = vert_pos(idx2, vt, ctab, r, v);
      e = make_float4(P.x, P.y, P.z, __fadd_rn(__fadd_rn(__fmul_rn(P.x, P.x), __fmul_rn(P.y, P.y)), __fmul_rn(P.z, P.z)));
      sw = ro[roi].nv >= p.sweep_min;
      if (sw) f2 = pair_f3(vert_pos(idx2, vt, ctab, r, ro[roi].v0 + (long long)(sweep[roi] & 0xffffffffull)), P);
    }
    if (__any_sync(0xffffffffu, sw)) sweep_step(acc, p.n > 1, sw, roi, f2, 0u, nullptr, ps);
    const RoiDiam& r = rd[roi];
    long long key[4];
    unsigned int peers[4];
    int base[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool use = v < n && (k == 0 || r.planes);
      key[k] = use ? (k == 0 ? key_of(r, q, 0) : plane_key(r, q, k, v, vt, fs)) : -1;
      peers[k] = __match_any_sync(0xffffffffu, key[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      base[k] = 0;
      if (key[k] >= 0 && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(&cursor[key[k]], __popc(peers[k]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int b = __shfl_sync(0xffffffffu, base[k], __ffs(peers[k]) - 1);
      if (key[k] >= 0) {
        const long long slot = offs[key[k]] + b + __popc(peers[k] & ((1u << lane) - 1u));
        sorted[slot] = e;
        ids[slot] = (int)v;
      }
    }
  }
  sweep_finish(acc, p.n == 1 && blockIdx.x * (long long)blockDim.x < n ? 0 : -1, &s_key, nullptr, ps);
}

// Exclusive scan of the key counts to global offsets, one kernel with a
// decoupled look-back over chunks of kScanBlock keys (4 per thread).
constexpr int kScanBlock = 4096;
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_xscan(const int* in, long long n, int nchunks,
                                                        long long* out, ScanTile<1>* tiles,
                                                        unsigned int* tick,
                                                        unsigned int* status) {
  pdl_enter();
  __shared__ long long ws[32];
  __shared__ long long s_ex;
  __shared__ int s_c;
  if (threadIdx.x == 0) s_c = (int)atomicAdd(tick, 1u);
  __syncthreads();
  const int c = s_c;
  const long long i0 = (long long)c * kScanBlock + 4 * threadIdx.x;
  long long v[4];
  long long own = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = i0 + k < n ? in[i0 + k] : 0;
    own += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc = own;
  for (int off = 1; off < 32; off <<= 1) {
    const long long o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  long long wb = 0, tot = 0;
  for (int k = 0; k < kScanThreads / 32; ++k) {
    if (k < wid) wb += ws[k];
    tot += ws[k];
  }
  if (threadIdx.x == 0) scan_publish(&tiles[c], &tot, c == 0 ? 2ull : 1ull);
  if (wid == 0) {
    long long e = 0;
    if (c > 0) {
      scan_lookback(tiles, c, &e, status);
      if (lane == 0) {
        const long long incl = e + tot;
        scan_publish(&tiles[c], &incl, 2ull);
      }
    }
    if (lane == 0) s_ex = e;
  }
  __syncthreads();
  long long x = s_ex + wb + inc - own;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (i0 + k < n) out[i0 + k] = x;
    x += v[k];
  }
}


// ---- 2. problems and tiles --------------------------------------------------------
// One lane per candidate problem: the 3D problem of every ROI (items 0..n-1)
// and every plane of every ROI (items n..).  A problem with >= 2 vertices
// takes a slot, and -- in one 64-bit atomic, so both ranges follow the same
// order -- a contiguous run of tiles and of seed/cull chunks (the order of
// problems does not affect any result).  Row i of a problem with nt tiles
// scans tiles i..nt-1 in ceil((nt - i) / kChunk) chunks.  The setup writes
// each tile's problem slot only (into chunk0); the tile kernel, one warp per
// tile, builds the tile record and its first chunk from the problem, so a
// problem with thousands of tiles is not written by one warp.
__device__ __forceinline__ int roi_of_plane(const RoiDiam* rd, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rd[mid].plane0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// sum over k = 1..m of ceil(k / kChunk): the chunks of the last m rows.
__device__ __forceinline__ long long chunks_upto(long long m) {
  const long long q = m / kChunk, r = m % kChunk;
  return kChunk * q * (q + 1) / 2 + r * (q + 1);
}

__global__ void k_setup(const RoiDiam* rd, Params p, const long long* offs,
                        Problem* probs, int* chunk0, Counters* cnt, FracState fs) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long items = p.n + p.nplanes + (fs.hkey ? fs.gcap : 0);
  const long long ngroups = fs.hkey ? min((long long)cnt->n_groups, fs.gcap) : 0;
  for (long long r0 = 0; r0 < items; r0 += nwarps * 32) {
    // one lane per candidate problem, dealt with a stride of the warp count,
    // so the ROIs' 3D problems (the largest) go to different warps
    const long long it = r0 + lane * nwarps + warp;
    int roi = 0, axis = -1;
    long long beg = 0, len = 0;
    if (it < items) {
      long long k0, k1;
      if (it < p.n) {
        roi = (int)it;
        const RoiDiam& r = rd[roi];
        k0 = r.key0;
        k1 = r.key0 + r.C3;
      } else if (it >= p.n + p.nplanes) {  // a soft map's plane off the grid planes
        const long long g = it - p.n - p.nplanes;
        k0 = k1 = 0;
        if (g < ngroups) {
          roi = fs.gra[g] >> 2;
          axis = fs.gra[g] & 3;
          k0 = fs.fbase + g;
          k1 = k0 + 1;
        }
      } else {
        const long long g = it - p.n;
        roi = roi_of_plane(rd, p.n, g);
        const RoiDiam& r = rd[roi];
        const long long l = g - r.plane0;
        const long long nz2 = 2LL * r.nz + 1, ny2 = 2LL * r.ny + 1;
        if (l < nz2) {
          axis = 2; k0 = r.key0 + r.S0 + l * r.PX * r.PY; k1 = k0 + (long long)r.PX * r.PY;
        } else if (l < nz2 + ny2) {
          axis = 1; k0 = r.key0 + r.S1 + (l - nz2) * r.PX * r.PZ; k1 = k0 + (long long)r.PX * r.PZ;
        } else {
          axis = 0; k0 = r.key0 + r.S2 + (l - nz2 - ny2) * r.PY * r.PZ; k1 = k0 + (long long)r.PY * r.PZ;
        }
      }
      beg = offs[k0];
      len = offs[k1] - beg;
    }
    const bool use = len >= 2;
    const unsigned int um = __ballot_sync(0xffffffffu, use);
    if (um == 0) continue;  // warp-uniform
    // warp-aggregated allocation of slots, walked tiles and chunks, and fine
    // tiles.  A problem of kBigTiles tiles or more takes two slots: its fine
    // problem (tiles in the fine region, never walked) and its coarse problem
    // (walked, one tile per kCoarse fine tiles).
    const int ntf = use ? (int)((len + p.TS - 1) / p.TS) : 0;
    const bool big = ntf >= kBigTiles;
    const int nt = big ? (ntf + kCoarse - 1) / kCoarse : ntf;  // walked tiles
    const int nslot = use ? (big ? 2 : 1) : 0;
    const int nfin = big ? ntf : 0;
    const long long S = use ? chunks_upto(nt) : 0;
    const unsigned long long add = use ? ((unsigned long long)S << 32) + (unsigned long long)nt : 0ull;
    unsigned long long inc = add;
    int sinc = nslot, finc = nfin;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, off);
      const int os = __shfl_up_sync(0xffffffffu, sinc, off), of = __shfl_up_sync(0xffffffffu, finc, off);
      if (lane >= off) { inc += o; sinc += os; finc += of; }
    }
    const unsigned long long total = __shfl_sync(0xffffffffu, inc, 31);
    const int stotal = __shfl_sync(0xffffffffu, sinc, 31), ftotal = __shfl_sync(0xffffffffu, finc, 31);
    int slot0 = 0;
    unsigned int fine0 = 0;
    unsigned long long old0 = 0;
    if (lane == 0) {
      slot0 = atomicAdd(&cnt->n_problems, stotal);
      old0 = atomicAdd(&cnt->alloc, total);
      if (ftotal) fine0 = atomicAdd(&cnt->alloc_fine, (unsigned int)ftotal);
    }
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    old0 = __shfl_sync(0xffffffffu, old0, 0);
    fine0 = __shfl_sync(0xffffffffu, fine0, 0);
    unsigned long long tp = use ? (unsigned long long)nt * (nt + 1) / 2 : 0ull;
    for (int off = 16; off > 0; off >>= 1) tp += __shfl_xor_sync(0xffffffffu, tp, off);
    if (lane == 0) atomicAdd((unsigned long long*)&cnt->n_pairs, tp);
    const int slot = slot0 + sinc - nslot;
    const long long fb = (long long)fine0 + finc - nfin;  // first fine tile (region offset)
    const unsigned long long old = old0 + (inc - add);
    const long long tb = (long long)(old & 0xffffffffull);
    const long long cb = (long long)(old >> 32);
    const bool ok = use && slot + nslot <= p.max_problems && tb + nt <= p.max_tiles && fb + nfin <= p.max_fine;
    // more than 2^31 chunks in one batch (about 740k tiles in one problem):
    // reported, and the chunk walk stays inside the tile array
    const bool ovf = ok && cb + S > (long long)INT_MAX;
    if ((use && !ok) || ovf) atomicOr(&cnt->status, DEV_ERR_PROBCAP);
    const int q = slot_of_axis(axis);
    const int wslot = big ? slot + 1 : slot;  // slot of the walked problem
    if (ok) {
      Problem pr;
      pr.axis = axis; pr.beg = (int)beg; pr.len = (int)len; pr.tile_beg = (int)tb; pr.roi = roi; pr.q = q;
      pr.nt = nt; pr.fine = -1;
      pr.chunk_end = ovf ? -1 : cb + S;
      if (big) {
        Problem f = pr;
        f.tile_beg = (int)(p.max_tiles + fb);
        f.nt = ntf;
        f.fine = -2;
        f.chunk_end = 0;
        probs[slot] = f;
        pr.fine = f.tile_beg;
      }
      probs[wslot] = pr;
    }
    // the warp marks the tiles of each accepted problem with its slot
    unsigned int wm = __ballot_sync(0xffffffffu, ok);
    while (wm) {
      const int src = __ffs(wm) - 1;
      wm &= wm - 1;
      const int s_slot = __shfl_sync(0xffffffffu, wslot, src), s_nt = __shfl_sync(0xffffffffu, nt, src);
      const long long s_tb = __shfl_sync(0xffffffffu, tb, src);
      for (int t = lane; t < s_nt; t += 32) chunk0[s_tb + t] = s_slot;
      const int s_nf = __shfl_sync(0xffffffffu, nfin, src);
      const long long s_fb = __shfl_sync(0xffffffffu, fb, src);
      for (int t = lane; t < s_nf; t += 32) chunk0[p.max_tiles + s_fb + t] = s_slot - 1;
    }
  }
}

// The box of every coarse tile as the union of its fine tiles' boxes (one
// warp per walked tile, grid-stride).
__device__ __noinline__ void coarse_boxes(const Tile* tiles, int nt, float4* box) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long ti = warp; ti < nt; ti += nwarps) {
    const int nf = tiles[ti].nfine;
    if (nf == 0) continue;  // warp-uniform
    const int f0 = tiles[ti].fine0;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (lane < nf) {
      const float4 l4 = box[2 * (f0 + lane)], h4 = box[2 * (f0 + lane) + 1];
      lo[0] = l4.x; lo[1] = l4.y; lo[2] = l4.z;
      hi[0] = h4.x; hi[1] = h4.y; hi[2] = h4.z;
    }
    for (int off = 16; off > 0; off >>= 1)
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
        hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
      }
    if (lane == 0) {
      box[2 * ti] = make_float4(lo[0], lo[1], lo[2], 0.f);
      box[2 * ti + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
}

// One warp per tile (walked tiles, then the fine region): its record and
// first seed/cull chunk, the bounding box of its FP32 positions (coarse
// tiles: later, from their fine tiles), and its first vertex.
__global__ void k_tile_box(const float4* sorted, const Problem* probs, Params p,
                           const Counters* cnt, Tile* tiles, int* chunk0,
                           float4* box, float4* rep) {
  pdl_enter();
  const int nt = (int)min((long long)(cnt->alloc & 0xffffffffull), p.max_tiles);
  const int nf = (int)min((long long)cnt->alloc_fine, p.max_fine);
  const int np = (int)min((long long)cnt->n_problems, p.max_problems);
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = warp; k < (long long)nt + nf; k += nwarps) {
    const long long ti = k < nt ? k : p.max_tiles + (k - nt);
    const int slot = chunk0[ti];  // the problem's slot, from the setup
    if ((unsigned int)slot >= (unsigned int)np) continue;  // warp-uniform; not reached (tiles never outrun problems)
    const Problem pr = probs[slot];
    const int t = (int)(ti - pr.tile_beg);  // tile within its problem
    if (t < 0 || t >= pr.nt) continue;      // warp-uniform; as above
    const bool coarse = pr.fine >= 0;
    const int span = coarse ? kCoarse * p.TS : p.TS;
    Tile tl;
    tl.problem = slot;
    tl.beg = pr.beg + t * span;
    tl.len = min(span, pr.len - t * span);
    tl.tile_end = pr.tile_beg + pr.nt;
    tl.roi = pr.roi;
    tl.q = pr.q;
    tl.fine0 = coarse ? pr.fine + t * kCoarse : 0;
    tl.nfine = coarse ? min(kCoarse, (pr.len + p.TS - 1) / p.TS - t * kCoarse) : 0;
    __syncwarp();  // every lane has read the slot before lane 0 replaces it
    if (lane == 0) {
      tiles[ti] = tl;
      if (k < nt) chunk0[ti] = pr.chunk_end < 0 ? INT_MAX : (int)(pr.chunk_end - chunks_upto(pr.nt - t));
      rep[ti] = sorted[tl.beg];
    }
    if (coarse) continue;  // warp-uniform
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = lane; i < tl.len; i += 32) {
      const float4 v = sorted[tl.beg + i];
      lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
      hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
    }
    for (int off = 16; off > 0; off >>= 1)
      for (int k2 = 0; k2 < 3; ++k2) {
        lo[k2] = fminf(lo[k2], __shfl_xor_sync(0xffffffffu, lo[k2], off));
        hi[k2] = fmaxf(hi[k2], __shfl_xor_sync(0xffffffffu, hi[k2], off));
      }
    if (lane == 0) {
      box[2 * ti] = make_float4(lo[0], lo[1], lo[2], 0.f);
      box[2 * ti + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
}

// ---- 3. seed and cull over (tile row, chunk) items ----------------------------------
// The items of all problems are numbered 0..K-1 in tile order (chunk0[t] is
// the first item of tile row t, non-decreasing).  Each warp takes an equal
// contiguous range of items, finds its first row with a 32-way search and
// then walks forward.

__device__ __forceinline__ int warp_find_row(const int* chunk0, int nt, long long k) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = nt - 1;  // chunk0[lo] <= k; the row is in [lo, hi]
  while (hi > lo) {         // warp-uniform; the range shrinks every step
    const long long span = hi - lo;
    const int pos = lo + (int)((span * (lane + 1) + 31) / 32);  // lane 31 probes hi
    const unsigned int m = __ballot_sync(0xffffffffu, (long long)chunk0[pos] <= k);
    if (m == 0) {
      hi = __shfl_sync(0xffffffffu, pos, 0) - 1;
    } else {
      const int l = 31 - __clz(m);
      const int plo = __shfl_sync(0xffffffffu, pos, l);
      const int pnext = __shfl_sync(0xffffffffu, pos, l < 31 ? l + 1 : 31);
      lo = plo;
      if (l < 31) hi = pnext - 1;
    }
  }
  return lo;
}

struct ChunkWalk {
  long long k, kend;    // this warp's items
  int a;                // current tile row
  long long c0, next0;  // first item of row a and of row a + 1
};

__device__ __forceinline__ bool walk_begin(ChunkWalk& w, const int* chunk0, int nt, long long K) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long per = (K + nwarps - 1) / nwarps;
  w.k = warp * per;
  w.kend = min(K, w.k + per);
  if (nt <= 0 || w.k >= w.kend) return false;
  w.a = warp_find_row(chunk0, nt, w.k);
  w.c0 = chunk0[w.a];
  w.next0 = w.a + 1 < nt ? (long long)chunk0[w.a + 1] : LLONG_MAX;
  return true;
}

// Next row's entries, loaded one row ahead (every row has at least one item,
// so the walk moves at most one row per item).
struct RowAhead {
  Tile t;
  float4 v0, v1;    // seed: representative; cull: box
  long long next1;  // first item of the row after it
};

__device__ __forceinline__ void row_ahead(RowAhead& r, const Tile* tiles, const float4* v, int stride,
                                          const int* chunk0, int nt, int a) {
  if (a + 1 < nt) {
    r.t = tiles[a + 1];
    r.v0 = v[stride * (a + 1)];
    if (stride == 2) r.v1 = v[2 * (a + 1) + 1];
    r.next1 = a + 2 < nt ? (long long)chunk0[a + 2] : LLONG_MAX;
  }
}

__device__ __forceinline__ void seed_flush(float m, int fam, ProblemState* ps) {
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&ps[fam].F, __float_as_uint(m));
}

// Seed: the pairs of tile representatives (first vertices) in every tile
// pair of a problem, plus each tile's first-last pair, are actual vertex
// pairs, so their largest f is a valid starting F.  Before walking, the
// blocks form the coarse tiles' boxes; the block that finishes last turns
// every family's F into T(F) for the cull.  Five blocks per SM (48
// registers): more resident warps for this latency-bound walk measured
// faster than four or six.
__global__ void __launch_bounds__(256, 5) k_seed(const float4* sorted, const float4* rep, Params p,
                       const Tile* tiles, const int* chunk0, Counters* cnt,
                       ProblemState* ps, const RoiDiam* rd, float4* box) {
  pdl_enter();
  __shared__ bool s_last;
  const unsigned long long alloc = cnt->alloc;
  const int nt = (int)min((long long)(alloc & 0xffffffffull), p.max_tiles);
  const long long K = min((long long)(alloc >> 32), (long long)INT_MAX);
  const int lane = threadIdx.x & 31;
  if (cnt->alloc_fine) coarse_boxes(tiles, nt, box);  // only when some problem is walked at two levels
  ChunkWalk w;
  if (walk_begin(w, chunk0, nt, K)) {  // warp-uniform
    Tile ta = tiles[w.a];
    float4 ra = rep[w.a];
    RowAhead nx;
    row_ahead(nx, tiles, rep, 1, chunk0, nt, w.a);
    float m = 0.0f;
    for (; w.k < w.kend; ++w.k) {
      if (w.k >= w.next0 && w.a + 1 < nt) {  // warp-uniform
        if (fam_of(nx.t.roi, nx.t.q) != fam_of(ta.roi, ta.q)) {  // one flush per family
          seed_flush(m, fam_of(ta.roi, ta.q), ps);
          m = 0.0f;
        }
        ++w.a;
        ta = nx.t;
        ra = nx.v0;
        w.c0 = w.next0;
        w.next0 = nx.next1;
        row_ahead(nx, tiles, rep, 1, chunk0, nt, w.a);
      }
      const long long c = w.k - w.c0;
      const long long b0 = w.a + c * kChunk;
      if (c == 0 && lane == 0) m = fmaxf(m, pair_f(ra, sorted[ta.beg + ta.len - 1]));
#pragma unroll
      for (int u = 0; u < kChunk / 32; ++u) {
        const long long b = b0 + 32 * u + lane;
        if (b < ta.tile_end) m = fmaxf(m, pair_f(ra, rep[b]));
      }
    }
    seed_flush(m, fam_of(ta.roi, ta.q), ps);
  }
  // the block that finishes last turns every family's F into T(F)
  __threadfence();  // this thread's seeds are visible before the block takes its ticket
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cnt->seed_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < 4 * p.n; i += blockDim.x)
    ps[i].T = __float_as_uint(threshold(__uint_as_float(__ldcg(&ps[i].F)), rd[i >> 2]));
}

// Cull: every tile pair (a, b >= a) of a problem whose box bound reaches
// T(F) goes to the work list, with both vertex ranges and the bound.  Four
// blocks per SM (64 registers): more resident warps for this latency-bound
// walk measured faster than the uncapped 76 registers, small spill included.
// The surviving pairs of one coarse row's chunk (bit l of m[u]: column
// b0 + 32 u + l) go to the refine list.
__device__ __noinline__ void cull_coarse(const Tile* tiles, const Params& p, Counters* cnt,
                                         RefineItem* refine, const Tile& ta, long long b0, int a,
                                         const unsigned int* m) {
  constexpr int U = kChunk / 32;
  const int lane = threadIdx.x & 31;
  int total = 0;
  for (int u = 0; u < U; ++u) total += __popc(m[u]);
  long long rbase = 0;
  if (lane == 0) rbase = (long long)atomicAdd(&cnt->n_refine, (unsigned int)total);
  rbase = __shfl_sync(0xffffffffu, rbase, 0);
  for (int u = 0; u < U; ++u) {
    if ((m[u] >> lane) & 1u) {
      const long long slot = rbase + __popc(m[u] & ((1u << lane) - 1u));
      const long long b = b0 + 32 * u + lane;
      if (slot < p.refine_cap) {
        const Tile tb = tiles[b];
        RefineItem ri;
        ri.fa = ta.fine0; ri.na = ta.nfine; ri.fb = tb.fine0; ri.nb = tb.nfine;
        ri.problem = ta.problem - 1; ri.roi = ta.roi; ri.q = ta.q; ri.same = b == a;
        refine[slot] = ri;
      } else {
        atomicOr(&cnt->status, DEV_ERR_WORKCAP);
      }
    }
    rbase += __popc(m[u]);
  }
}

__global__ void __launch_bounds__(256, 4) k_cull(const Tile* tiles, const float4* box, Params p,
                       const int* chunk0, Counters* cnt, const ProblemState* ps,
                       WorkItem* work, RefineItem* refine) {
  pdl_enter();
  const unsigned long long alloc = cnt->alloc;
  const int nt = (int)min((long long)(alloc & 0xffffffffull), p.max_tiles);
  const long long K = min((long long)(alloc >> 32), (long long)INT_MAX);
  const int lane = threadIdx.x & 31;
  constexpr int U = kChunk / 32;
  ChunkWalk w;
  if (!walk_begin(w, chunk0, nt, K)) return;
  Tile ta = tiles[w.a];
  float4 alo = box[2 * w.a], ahi = box[2 * w.a + 1];
  int fam = fam_of(ta.roi, ta.q);
  float T = __uint_as_float(ps[fam].T);
  RowAhead nx;
  row_ahead(nx, tiles, box, 2, chunk0, nt, w.a);
  for (; w.k < w.kend; ++w.k) {
    if (w.k >= w.next0 && w.a + 1 < nt) {  // warp-uniform
      ++w.a;
      ta = nx.t;
      alo = nx.v0;
      ahi = nx.v1;
      w.c0 = w.next0;
      w.next0 = nx.next1;
      row_ahead(nx, tiles, box, 2, chunk0, nt, w.a);
      if (fam_of(ta.roi, ta.q) != fam) {
        fam = fam_of(ta.roi, ta.q);
        T = __uint_as_float(ps[fam].T);
      }
    }
    const long long b0 = w.a + (w.k - w.c0) * kChunk;
    bool keep[U];
    float ub[U];
    unsigned int m[U];
    int total = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long b = b0 + 32 * u + lane;
      keep[u] = false;
      ub[u] = 0.0f;
      if (b < ta.tile_end) {
        ub[u] = box_ub(alo, ahi, box[2 * b], box[2 * b + 1]);
        keep[u] = ub[u] >= T;
      }
      m[u] = __ballot_sync(0xffffffffu, keep[u]);
      total += __popc(m[u]);
    }
    if (total == 0) continue;  // warp-uniform
    if (ta.nfine > 0) {  // a coarse row: its surviving pairs are refined by the next kernel
      cull_coarse(tiles, p, cnt, refine, ta, b0, w.a, m);
      continue;
    }
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd((unsigned long long*)&cnt->n_work, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (keep[u]) {
        const long long slot = base + __popc(m[u] & ((1u << lane) - 1u));
        if (slot < p.work_cap) {
          const Tile tb = tiles[b0 + 32 * u + lane];
          WorkItem it;
          it.problem = ta.problem; it.roi = ta.roi; it.q = ta.q;
          it.abeg = ta.beg; it.alen = ta.len; it.bbeg = tb.beg; it.blen = tb.len;
          it.ub = ub[u];
          work[slot] = it;
        } else {
          atomicOr(&cnt->status, DEV_ERR_WORKCAP);
        }
      }
      base += __popc(m[u]);
    }
  }
}

// Refinement of the surviving coarse tile pairs, one warp per pair: lane l
// holds the boxes of fine tile l of both coarse tiles in registers, and the
// warp tests each fine tile of the first (broadcast by shuffles) against the
// lanes' fine tiles of the second (only b >= a within one coarse tile).
// Surviving fine pairs go to the work list.
__global__ void k_refine(const Tile* tiles, const float4* box, Params p,
                         Counters* cnt, const ProblemState* ps,
                         const RefineItem* refine, WorkItem* work) {
  pdl_enter();
  const long long nr = min((long long)cnt->n_refine, p.refine_cap);
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = warp; k < nr; k += nwarps) {
    const RefineItem ri = refine[k];
    const float T = __uint_as_float(ps[fam_of(ri.roi, ri.q)].T);
    const bool ha = lane < ri.na, hb = lane < ri.nb;
    const int a_own = ri.fa + lane, b = ri.fb + lane;
    float4 alo = make_float4(0.f, 0.f, 0.f, 0.f), ahi = alo, blo = alo, bhi = alo;
    int bbeg = 0, blen = 0;
    if (ha) {
      alo = box[2 * a_own];
      ahi = box[2 * a_own + 1];
    }
    if (hb) {
      blo = box[2 * b];
      bhi = box[2 * b + 1];
      bbeg = tiles[b].beg;
      blen = tiles[b].len;
    }
    unsigned int am = 0u;  // fine tiles of the first coarse tile whose pair with this lane's tile survives
    for (int ia = 0; ia < ri.na; ++ia) {  // warp-uniform
      const float4 l4 = make_float4(__shfl_sync(0xffffffffu, alo.x, ia), __shfl_sync(0xffffffffu, alo.y, ia),
                                    __shfl_sync(0xffffffffu, alo.z, ia), 0.f);
      const float4 h4 = make_float4(__shfl_sync(0xffffffffu, ahi.x, ia), __shfl_sync(0xffffffffu, ahi.y, ia),
                                    __shfl_sync(0xffffffffu, ahi.z, ia), 0.f);
      if (hb && (!ri.same || lane >= ia)) {
        if (box_ub(l4, h4, blo, bhi) >= T) am |= 1u << ia;
      }
    }
    const int mine = __popc(am);
    int incl = mine;
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;  // warp-uniform
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd((unsigned long long*)&cnt->n_work, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0) + (incl - mine);
    for (unsigned int mm = am; mm; mm &= mm - 1, ++base) {
      const int ia = __ffs(mm) - 1;
      if (base < p.work_cap) {
        const int a = ri.fa + ia;
        const Tile ta = tiles[a];
        WorkItem it;
        it.problem = ri.problem; it.roi = ri.roi; it.q = ri.q;
        it.abeg = ta.beg; it.alen = ta.len; it.bbeg = bbeg; it.blen = blen;
        it.ub = box_ub(box[2 * a], box[2 * a + 1], blo, bhi);
        work[base] = it;
      } else {
        atomicOr(&cnt->status, DEV_ERR_WORKCAP);
      }
    }
  }
}

// ---- 4. pair kernel -----------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// B slices per warp unit: a unit is tile A of a work item against G
// consecutive 32-entry slices of its tile B.  Two slices share the staging
// and expansion of A; more would leave each warp too few units for a rising
// T to cull the later ones (T is read when a unit is staged and again before
// each slice).
template <int TS>
__host__ __device__ constexpr int pair_slices() {
  return 2;
}

// Dynamic shared memory of the pair kernel, per warp: tile A and the unit's
// B slices, double buffered, plus two duplicated B slices (32 B an entry).
template <int TS, int NT>
constexpr size_t pair_smem_bytes() {
  return (size_t)(NT / 32) * (2 * TS * sizeof(float4) + 2 * 32 * pair_slices<TS>() * sizeof(float4) +
                              2 * 2 * 32 * sizeof(ulonglong2));
}

// One warp unit: tile A and the B slices s0 .. s0 + G - 1 of a work item into
// the warp's own shared-memory buffers.  Entries past a tile's length repeat
// its last vertex (a real vertex, so maxima are unaffected); slices wholly
// past it are not copied.
template <int TS, int G>
__device__ __forceinline__ void stage_unit(float4* sA, float4* sB, const float4* sorted, const WorkItem& w, int s0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < TS / 32; ++r) cp_async16(&sA[lane + 32 * r], &sorted[w.abeg + min(lane + 32 * r, w.alen - 1)]);
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (32 * (s0 + g) < w.blen) cp_async16(&sB[32 * g + lane], &sorted[w.bbeg + min(32 * (s0 + g) + lane, w.blen - 1)]);
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Every warp works on its own over units u, u + W, u + 2W, ... (u its global
// warp index, W the number of warps; the warps of a CTA take neighbouring
// units, so tiles shared between them come from L1).  It stages the next
// unit with cp.async while it evaluates the current one (no block barrier
// anywhere) and skips a unit whose bound is below the current T.  Otherwise
// it expands tile A once (lane l holds the A entries l, l + 32, ...), works
// through the unit's B slices (T is read again before each, so a unit stops
// once T passes its bound), stores each slice maximum, and raises F (and T)
// when the unit's maximum beats F.  slicemax[slice] < 0 marks a skipped or
// empty slice.
template <int TS, int NT>
__global__ void __launch_bounds__(NT) k_pairs(const float4* sorted, const WorkItem* work,
                                              Params p, const RoiDiam* rd, Counters* cnt,
                                              ProblemState* ps, float* slicemax) {
  pdl_enter();
  constexpr int RA = TS / 32;  // A entries per lane, and B slices per tile pair
  constexpr int G = pair_slices<TS>();
  constexpr int UPI = RA / G;  // units per work item
  constexpr int NWARP = NT / 32;
  static_assert(RA % G == 0 && RA % 2 == 0, "slices per unit");
  extern __shared__ __align__(16) unsigned char pair_smem[];
  float4(*sA)[2][TS] = reinterpret_cast<float4(*)[2][TS]>(pair_smem);
  float4(*sB)[2][32 * G] = reinterpret_cast<float4(*)[2][32 * G]>(pair_smem + NWARP * 2 * TS * sizeof(float4));
  // one slice's B, duplicated: (x,x | y,y), (z,z | n,n)
  ulonglong2(*sB2)[2][2][32] = reinterpret_cast<ulonglong2(*)[2][2][32]>(
      pair_smem + NWARP * 2 * (TS + 32 * G) * sizeof(float4));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long nunits = min(cnt->n_work, p.work_cap) * UPI;
  const long long W = (long long)gridDim.x * NWARP;
  long long t_cur = (long long)blockIdx.x * NWARP + wid;
  if (t_cur >= nunits) return;  // warp-uniform
  WorkItem w_cur = work[t_cur / UPI];
  stage_unit<TS, G>(sA[wid][0], sB[wid][0], sorted, w_cur, (int)(t_cur % UPI) * G);
  cp_async_commit();
  unsigned long long ft_cur = *(volatile unsigned long long*)&ps[fam_of(w_cur.roi, w_cur.q)];
  long long t_nxt = t_cur + W;
  WorkItem w_nxt = t_nxt < nunits ? work[t_nxt / UPI] : w_cur;
  int buf = 0;
  unsigned long long n_items = 0, n_pairs = 0;
  // duplicate B entry `lane` of slice g into sB2[d]
  auto dup = [&](int g, int d) {
    const float4 b = sB[wid][buf][32 * g + lane];
    sB2[wid][d][0][lane] = make_ulonglong2(pk2(b.x, b.x), pk2(b.y, b.y));
    sB2[wid][d][1][lane] = make_ulonglong2(pk2(b.z, b.z), pk2(b.w, b.w));
  };
  while (true) {
    const bool has_next = t_nxt < nunits;
    __syncwarp();  // every lane is done with the other buffer
    unsigned long long ft_nxt = ft_cur;
    if (has_next) {
      stage_unit<TS, G>(sA[wid][buf ^ 1], sB[wid][buf ^ 1], sorted, w_nxt, (int)(t_nxt % UPI) * G);
      ft_nxt = *(volatile unsigned long long*)&ps[fam_of(w_nxt.roi, w_nxt.q)];
    }
    cp_async_commit();
    const long long t_nn = t_nxt + W;
    const WorkItem w_nn = t_nn < nunits ? work[t_nn / UPI] : w_nxt;
    cp_async_wait<1>();  // this lane's copies of the current unit have landed
    __syncwarp();        // ... and every lane's
    const float F = __uint_as_float((unsigned int)ft_cur), T = __uint_as_float((unsigned int)(ft_cur >> 32));
    const long long item = t_cur / UPI;
    const int s0 = (int)(t_cur % UPI) * G;
    const int ns = min(G, (w_cur.blen + 31) / 32 - s0);  // non-empty slices of the unit
    float um = -1.0f;
    int ne = 0;  // slices evaluated
    if (!(w_cur.ub < T) && ns > 0) {
      // A entries r and r + 1 packed per coordinate; B duplicated, so three
      // f32x2 FMAs give two pairs (the same operations, in the same order, as
      // pair_h; pair_g's final add of n_a is applied once per slice maximum)
      unsigned long long ax[RA / 2], ay[RA / 2], az[RA / 2], an[RA / 2];
#pragma unroll
      for (int r = 0; r < RA; r += 2) {
        const float4 a0 = expand_a(sA[wid][buf][lane + 32 * r]), a1 = expand_a(sA[wid][buf][lane + 32 * (r + 1)]);
        ax[r / 2] = pk2(a0.x, a1.x); ay[r / 2] = pk2(a0.y, a1.y);
        az[r / 2] = pk2(a0.z, a1.z); an[r / 2] = pk2(a0.w, a1.w);
      }
      dup(0, 0);
      __syncwarp();
#pragma unroll 1
      for (int g = 0; g < ns; ++g) {
        // T for the next slice, read now and used after this slice's loop
        const unsigned int tn = g + 1 < ns ? *(volatile unsigned int*)&ps[fam_of(w_cur.roi, w_cur.q)].T : 0u;
        if (g + 1 < ns) dup(g + 1, (g + 1) & 1);  // read only after the barrier below
        const ulonglong2* bxy = sB2[wid][g & 1][0];
        const ulonglong2* bzn = sB2[wid][g & 1][1];
        // h = fma(-2a_x, b_x, fma(-2a_y, b_y, fma(-2a_z, b_z, n_b))) per pair,
        // its maximum over the slice per A entry, and n_a added once at the end
        float mx[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) mx[r] = -FLT_MAX;
#pragma unroll 4
        for (int j = 0; j < 32; j += 2) {
          const ulonglong2 p0 = bxy[j], p1 = bzn[j], q0 = bxy[j + 1], q1 = bzn[j + 1];
#pragma unroll
          for (int h = 0; h < RA / 2; ++h) {
            unsigned long long g0 = fma2(az[h], p1.x, p1.y), g1 = fma2(az[h], q1.x, q1.y);
            g0 = fma2(ay[h], p0.y, g0); g1 = fma2(ay[h], q0.y, g1);
            g0 = fma2(ax[h], p0.x, g0); g1 = fma2(ax[h], q0.x, g1);
            float g00, g01, g10, g11;
            unpk2(g0, g00, g01);
            unpk2(g1, g10, g11);
            mx[2 * h] = max3f(mx[2 * h], g00, g10);
            mx[2 * h + 1] = max3f(mx[2 * h + 1], g01, g11);
          }
        }
        __syncwarp();  // slice g is read, slice g + 1's duplicate is visible
        float m = 0.0f;  // f is never below 0 in exact arithmetic; a rounded value below counts as 0
#pragma unroll
        for (int h = 0; h < RA / 2; ++h) {
          float g0, g1;
          unpk2(add2(an[h], pk2(mx[2 * h], mx[2 * h + 1])), g0, g1);
          m = max3f(m, g0, g1);
        }
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) {
          slicemax[item * RA + s0 + g] = m;
          n_pairs += (unsigned long long)w_cur.alen * (unsigned long long)min(32, w_cur.blen - 32 * (s0 + g));
        }
        um = fmaxf(um, m);
        ne = g + 1;
        if (w_cur.ub < __uint_as_float(tn)) break;  // T has passed the bound: skip the unit's other slices
      }
      if (lane == 0) {
        if (um > F) {  // fire and forget: T(F) is monotone, so the largest maximum wins both
          atomicMax(&ps[fam_of(w_cur.roi, w_cur.q)].F, __float_as_uint(um));
          atomicMax(&ps[fam_of(w_cur.roi, w_cur.q)].T, __float_as_uint(threshold(um, rd[w_cur.roi])));
        }
        n_items += s0 == 0;
      }
    }
    if (lane < G && lane >= ne) slicemax[item * RA + s0 + lane] = -1.0f;
    if (!has_next) break;
    t_cur = t_nxt;
    w_cur = w_nxt;
    ft_cur = ft_nxt;
    t_nxt = t_nn;
    w_nxt = w_nn;
    buf ^= 1;
  }
  cp_async_wait<0>();
  if (lane == 0 && n_pairs) {
    atomicAdd(&cnt->items_evaluated, n_items);
    atomicAdd(&cnt->pairs_evaluated, n_pairs);
  }
}

// Slices whose maximum reaches their problem's final T, listed compactly
// (one lane per slice).
template <int TS>
__global__ void k_cand_list(const WorkItem* work, const float* slicemax, Params p,
                            Counters* cnt, const ProblemState* ps, int* hits) {
  pdl_enter();
  constexpr int RA = TS / 32;
  const long long nslices = min(cnt->n_work, p.work_cap) * RA;
  const int lane = threadIdx.x & 31;
  for (long long s0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; s0 < nslices;
       s0 += (long long)gridDim.x * blockDim.x) {
    const long long sl = s0 + lane;
    bool hit = false;
    if (sl < nslices) {
      const float m = slicemax[sl];
      if (m >= 0.0f) {
        const WorkItem& w = work[sl / RA];
        hit = m >= __uint_as_float(ps[fam_of(w.roi, w.q)].T);
      }
    }
    const unsigned int hm = __ballot_sync(0xffffffffu, hit);
    if (hm == 0) continue;
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd((unsigned long long*)&cnt->n_hits, (unsigned long long)__popc(hm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) hits[base + __popc(hm & ((1u << lane) - 1u))] = (int)sl;
  }
}

// Candidates: one warp per listed slice rescans it (A entries in registers,
// the 32 B entries one per lane, broadcast by shuffles) and lists its pairs
// with f >= T.  A warp stages its candidates in shared memory and reserves
// list slots 33..64 at a time, so the list counter sees few atomics.
constexpr int kCandThreads = 256;
template <int TS>
__global__ void __launch_bounds__(kCandThreads) k_cand(const float4* sorted,
                                                       const WorkItem* work, const int* hits,
                                                       Params p, Counters* cnt,
                                                       const ProblemState* ps, Cand* cand) {
  pdl_enter();
  constexpr int RA = TS / 32;
  const long long nh = cnt->n_hits;
  const int lane = threadIdx.x & 31;
  __shared__ Cand s_cb[kCandThreads / 32][64];
  Cand* cb = s_cb[threadIdx.x >> 5];
  int cbn = 0;  // staged candidates (warp-uniform)
  auto cflush = [&]() {
    __syncwarp();
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd((unsigned long long*)&cnt->n_cand, (unsigned long long)cbn);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < cbn; i += 32) {
      if (base + i < p.cand_cap) cand[base + i] = cb[i];
      else atomicOr(&cnt->status, DEV_ERR_CANDCAP);
    }
    __syncwarp();
    cbn = 0;
  };
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  // the next hit's slice and work item are loaded while the current one is rescanned
  int sl_nxt = warp < nh ? hits[warp] : 0;
  WorkItem w_nxt;
  if (warp < nh) w_nxt = work[sl_nxt / RA];
  for (long long h = warp; h < nh; h += nwarps) {
    const int sl = sl_nxt;
    const WorkItem w = w_nxt;
    const float T = __uint_as_float(ps[fam_of(w.roi, w.q)].T);
    const int jb = (sl % RA) * 32;
    const bool same = w.abeg == w.bbeg;
    float4 a[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) a[r] = expand_a(sorted[w.abeg + min(lane + 32 * r, w.alen - 1)]);
    const float4 bl = sorted[w.bbeg + min(jb + lane, w.blen - 1)];
    if (h + nwarps < nh) {
      sl_nxt = hits[h + nwarps];
      w_nxt = work[sl_nxt / RA];
    }
    const int nj = min(32, w.blen - jb);
    for (int jj = 0; jj < nj; ++jj) {
      float4 b;
      b.x = __shfl_sync(0xffffffffu, bl.x, jj);
      b.y = __shfl_sync(0xffffffffu, bl.y, jj);
      b.z = __shfl_sync(0xffffffffu, bl.z, jj);
      b.w = __shfl_sync(0xffffffffu, bl.w, jj);
      const int j = jb + jj;
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        const int ia = lane + 32 * r;
        const bool c = ia < w.alen && (!same || ia < j) && pair_g(a[r], b) >= T;
        const unsigned int cm = __ballot_sync(0xffffffffu, c);
        if (cm == 0) continue;  // warp-uniform
        if (c) {
          Cand k;
          k.ea = w.abeg + ia; k.eb = w.bbeg + j; k.roi = w.roi; k.q = w.q;
          cb[cbn + __popc(cm & ((1u << lane) - 1u))] = k;
        }
        cbn += __popc(cm);
        if (cbn > 32) cflush();
      }
    }
  }
  if (cbn) cflush();
}

// ---- FP64 in place of the FP32 filter (the culled FP64 variant) ---------------------

// Every pair of every surviving work item in FP64 with the pinned formula:
// one warp per work item (re-culled against the current T first), the A
// entries' positions in registers (lane l holds entries l, l + 32, ...), the
// B entries staged 32 at a time in the warp's shared memory.  Each lane keeps
// its best (d2, i, j) key; the warp's best goes to the family's 128-bit key
// with one atomic and raises F to d2 rounded down (a value no larger than the
// FP64 maximum, so T(F) stays below every pair that attains it).
constexpr int kP64Threads = 256;
template <int TS>
__global__ void __launch_bounds__(kP64Threads) k_pairs64(const int* ids, const int16_t* idx2, const double* vt,
                                                         const WorkItem* work, Params p, const RoiDiam* rd,
                                                         const RoiOut* ro, Counters* cnt, ProblemState* ps,
                                                         Key128* keys) {
  pdl_enter();
  constexpr int RA = TS / 32;
  __shared__ double s_u[kP64Threads / 32][3][32];
  __shared__ int s_id[kP64Threads / 32][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long nitems = min(cnt->n_work, p.work_cap);
  const long long nwarps = (long long)gridDim.x * (kP64Threads / 32);
  unsigned long long n_items = 0, n_pairs = 0;
  for (long long it = (long long)blockIdx.x * (kP64Threads / 32) + wid; it < nitems; it += nwarps) {
    const WorkItem w = work[it];
    const int fam = fam_of(w.roi, w.q);
    if (w.ub < __uint_as_float(*(volatile unsigned int*)&ps[fam].T)) continue;  // warp-uniform
    const long long v0 = ro[w.roi].v0;
    const RoiDiam& r = rd[w.roi];
    const bool same = w.abeg == w.bbeg;
    double ua[RA][3];
    int ia[RA];
#pragma unroll
    for (int k = 0; k < RA; ++k) {
      const int e = lane + 32 * k;
      ia[k] = -1;
      if (e < w.alen) {
        const int id = ids[w.abeg + e];
        vertex_u(idx2, vt, id, ua[k]);
        ia[k] = id - (int)v0;
      }
    }
    Key128 best{0ull, 0ull};
    for (int jb = 0; jb < w.blen; jb += 32) {
      __syncwarp();
      if (jb + lane < w.blen) {
        const int id = ids[w.bbeg + jb + lane];
        double u[3];
        vertex_u(idx2, vt, id, u);
        s_u[wid][0][lane] = u[0];
        s_u[wid][1][lane] = u[1];
        s_u[wid][2][lane] = u[2];
        s_id[wid][lane] = id - (int)v0;
      }
      __syncwarp();
      const int nj = min(32, w.blen - jb);
      for (int jj = 0; jj < nj; ++jj) {
        const double bx = s_u[wid][0][jj], by = s_u[wid][1][jj], bz = s_u[wid][2][jj];
        const int jid = s_id[wid][jj];
#pragma unroll
        for (int k = 0; k < RA; ++k) {
          if (ia[k] < 0 || (same && lane + 32 * k >= jb + jj)) continue;
          const double d2 = pin_d2(ua[k][0], ua[k][1], ua[k][2], bx, by, bz, r.sx, r.sy, r.sz);
          const Key128 key = make_key(d2, min(ia[k], jid), max(ia[k], jid));
          if (key_gt(key, best)) best = key;
        }
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      Key128 o;
      o.lo = __shfl_xor_sync(0xffffffffu, best.lo, off);
      o.hi = __shfl_xor_sync(0xffffffffu, best.hi, off);
      if (key_gt(o, best)) best = o;
    }
    if (lane == 0) {
      ++n_items;
      n_pairs += same ? (unsigned long long)w.alen * (w.alen - 1) / 2 : (unsigned long long)w.alen * w.blen;
      if (best.hi | best.lo) {
        atomic_max_key(&keys[fam], best);
        const float Fn = __double2float_rd(__longlong_as_double((long long)best.hi));
        if (Fn > __uint_as_float(*(volatile unsigned int*)&ps[fam].F)) {
          atomicMax(&ps[fam].F, __float_as_uint(Fn));
          atomicMax(&ps[fam].T, __float_as_uint(threshold(Fn, r)));
        }
      }
    }
  }
  if (lane == 0 && n_pairs) {
    atomicAdd(&cnt->items_evaluated, n_items);
    atomicAdd(&cnt->pairs_evaluated, n_pairs);
  }
}

// The families' keys into the per-ROI results (d2 bits and (i << 32 | j)).
__global__ void k_keys_out(const Key128* keys, int n, DiamOut* out) {
  pdl_enter();
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < 4 * n; f += gridDim.x * blockDim.x) {
    const Key128 k = keys[f];
    if (k.hi | k.lo) {
      out[f >> 2].d2[f & 3] = k.hi;
      out[f >> 2].pair[f & 3] = ~k.lo;
    }
  }
}

// ---- 5. FP64 confirmation -------------------------------------------------------------

// The FP64 confirmation: every candidate's pinned FP64 d2 and its pair (ids
// local to the ROI, i < j) as one 128-bit key, raised into its (ROI,
// category) family with a compare-and-swap: the largest d2, then the
// smallest (i, j).  Every pair attaining the maximum is a candidate of its
// problem, so the family's key is the FP64 maximum with its tie-break.  The
// block that finishes last writes the keys into the per-ROI results and
// copies the counters.
__device__ void copy_stats(Counters* cnt, DiamStats* stats) {
  stats->problems = cnt->n_problems;
  stats->tiles = (long long)(cnt->alloc & 0xffffffffull) + (long long)cnt->alloc_fine;
  stats->tile_pairs = cnt->n_pairs;
  stats->work_items = cnt->n_work;
  stats->items_evaluated = (long long)cnt->items_evaluated;
  stats->pairs_evaluated = (long long)cnt->pairs_evaluated;
  stats->candidates = cnt->n_cand;
  stats->coarse_pairs = cnt->n_refine;
  stats->status |= cnt->status;
}

__global__ void k_confirm(const int* ids, const int16_t* idx2,
                          const double* vt, Params p, const RoiDiam* rd,
                          const RoiOut* ro, Counters* cnt, const Cand* cand,
                          Key128* keys, DiamOut* out, DiamStats* stats) {
  pdl_enter();
  __shared__ bool s_last;
  const long long nc = min(cnt->n_cand, p.cand_cap);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const Cand k = cand[c];
    const RoiDiam& r = rd[k.roi];
    int i = ids[k.ea], j = ids[k.eb];
    double ui[3], uj[3];
    vertex_u(idx2, vt, i, ui);
    vertex_u(idx2, vt, j, uj);
    const double d2 = pin_d2(ui[0], ui[1], ui[2], uj[0], uj[1], uj[2], r.sx, r.sy, r.sz);
    const int v0 = (int)ro[k.roi].v0;
    i -= v0;
    j -= v0;
    atomic_max_key(&keys[fam_of(k.roi, k.q)], make_key(d2, min(i, j), max(i, j)));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cnt->confirm_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int f = threadIdx.x; f < 4 * p.n; f += blockDim.x) {
    Key128 k;
    k.lo = __ldcg(&keys[f].lo);
    k.hi = __ldcg(&keys[f].hi);
    if (k.hi | k.lo) {
      out[f >> 2].d2[f & 3] = k.hi;
      out[f >> 2].pair[f & 3] = ~k.lo;
    }
  }
  if (threadIdx.x == 0) copy_stats(cnt, stats);
}

// Statistics only (the culled FP64 mode has no candidates).
__global__ void k_stats(Counters* cnt, DiamStats* stats) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) copy_stats(cnt, stats);
}

__global__ void k_diam_init(DiamOut* out, int n, ZeroSet zs, const RoiDiam* rd,
                            float* ctab, long long ntab) {
  pdl_enter();
  zero_ranges(zs);  // counters, statistics, key histogram and cursors, scan state
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int q = 0; q < 4; ++q) {
      out[i].d2[q] = 0ull;
      out[i].pair[q] = ~0ull;
    }
  // FP32 coordinate tables of the masks: the entry of doubled coordinate q
  // holds fl32((q / 2 - c) * s), the value the sorted entries carry
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ntab;
       e += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;  // last ROI whose tables start at or before e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rd[mid].tab0 <= e) lo = mid;
      else hi = mid - 1;
    }
    const RoiDiam& r = rd[lo];
    const long long l = e - r.tab0;
    const long long lx = 2LL * r.nx + 3, ly = 2LL * r.ny + 3;
    double c, sp;
    long long q;
    if (l < lx) { q = l - 2; c = r.cx; sp = r.sx; }
    else if (l < lx + ly) { q = l - lx - 2; c = r.cy; sp = r.sy; }
    else { q = l - lx - ly - 2; c = r.cz; sp = r.sz; }
    const double u = 0.5 * (double)q;
    ctab[e] = __double2float_rn((u - c) * sp);
  }
}

struct BestD {
  double d2;
  int i, j;
};

__device__ __forceinline__ bool better(double d2, int i, int j, const BestD& b) {
  if (b.i < 0) return i >= 0;
  if (i < 0) return false;
  if (d2 != b.d2) return d2 > b.d2;
  if (i != b.i) return i < b.i;
  return j < b.j;
}

template <class T>
T* carve(char*& cur, size_t n) {
  T* r = reinterpret_cast<T*>(cur);
  cur += (n * sizeof(T) + 255) & ~size_t(255);
  return r;
}

template <int TS, int NT>
rad_status launch_pairs(const float4* sorted, const WorkItem* work, const Params& p, const RoiDiam* rd, Counters* cnt,
                        ProblemState* ps, float* slicemax, int* hits, Cand* cand, int ctas, cudaStream_t st) {
  auto kp = k_pairs<TS, NT>;
  auto kl = k_cand_list<TS>;
  auto kc = k_cand<TS>;
  constexpr size_t smem = pair_smem_bytes<TS, NT>();
  {  // once per device; the first pass of a workspace runs eagerly, before any capture
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    RAD_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
      RAD_CUDA(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      done.fetch_or(bit);
    }
  }
  // at most one full wave: the units are dealt out to the grid's warps
  const int pgrid = std::min(ctas, wave_grid(kp, NT, 1LL << 30, smem));
  RAD_LAUNCH("diam_pairs_fp32", kp, pgrid, NT, smem, st, sorted, work, p, rd, cnt, ps, slicemax);
  RAD_LAUNCH("diam_cand_list", kl, wave_grid(kl, 256, num_sms() * 4), 256, 0, st, work, slicemax, p, cnt, ps, hits);
  RAD_LAUNCH("diam_pairs_cand", kc, wave_grid(kc, kCandThreads, num_sms() * 4), kCandThreads, 0, st, sorted, work,
             hits, p, cnt, ps, cand);
  return RAD_OK;
}

}  // namespace

// Entries of a mask ROI's FP32 coordinate tables: doubled coordinates
// q = -2 .. 2n (the vertices use -2 .. 2n - 1) per axis, x then y then z.
static long long coord_table_len(int nx, int ny, int nz) {
  return (2LL * nx + 3) + (2LL * ny + 3) + (2LL * nz + 3);
}

// Host-side per-ROI parameters of the diameter problems.
void plan_diam(const std::vector<Roi>& rois, bool soft, std::vector<RoiDiam>& rd, long long& nkeys, long long& ntab,
               long long& nplanes) {
  const rad_tuning_t& tu = tuning();
  rd.resize(rois.size());
  nkeys = 0;
  ntab = 0;
  nplanes = 0;
  const double u = ldexp(1.0, -24);
  for (size_t i = 0; i < rois.size(); ++i) {
    const Roi& g = rois[i];
    RoiDiam& p = rd[i];
    p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
    p.planes = 1;  // masks and soft maps: the planar diameters too
    p.cell_shift = tu.cell_shift;
    p.CX = ((2 * g.nx) >> p.cell_shift) + 1;
    p.CY = ((2 * g.ny) >> p.cell_shift) + 1;
    p.CZ = ((2 * g.nz) >> p.cell_shift) + 1;
    p.plane_shift = tu.cell_shift + 2;
    p.PX = ((2 * g.nx) >> p.plane_shift) + 1;
    p.PY = ((2 * g.ny) >> p.plane_shift) + 1;
    p.PZ = ((2 * g.nz) >> p.plane_shift) + 1;
    p.C3 = (long long)p.CX * p.CY * p.CZ;
    p.S0 = p.C3;
    p.S1 = p.S0 + (p.planes ? (2LL * g.nz + 1) * p.PX * p.PY : 0);
    p.S2 = p.S1 + (p.planes ? (2LL * g.ny + 1) * p.PX * p.PZ : 0);
    p.K = p.S2 + (p.planes ? (2LL * g.nx + 1) * p.PY * p.PZ : 0);
    p.key0 = nkeys;
    p.plane0 = nplanes;
    p.tab0 = soft ? -1 : ntab;
    if (!soft) ntab += coord_table_len(g.nx, g.ny, g.nz);
    nkeys += p.K;
    nplanes += p.planes ? (2LL * g.nx + 1) + (2LL * g.ny + 1) + (2LL * g.nz + 1) : 0;
    p.sx = g.sx; p.sy = g.sy; p.sz = g.sz;
    p.cx = 0.5 * (g.nx - 1); p.cy = 0.5 * (g.ny - 1); p.cz = 0.5 * (g.nz - 1);
    double R2 = 0.0;
    const int nn[3] = {g.nx, g.ny, g.nz};
    const double sp[3] = {g.sx, g.sy, g.sz};
    for (int k = 0; k < 3; ++k) {
      const double r = 0.5 * (nn[k] + 1) * sp[k];
      R2 += r * r;
    }
    // the larger coefficient of the two FP32 forms, doubled
    p.alpha = 2.0 * 5.1 * u + 1e-14;
    p.beta = 2.0 * 4.1 * u * sqrt(R2);
    p.gamma = 2.0 * std::max(20.2 * u * R2, 4.1 * u * u * R2);
  }
}

rad_status diam_run(int n, const RoiDiam* rd, const RoiOut* ro, const long long* nv_dev, long long nv_cap,
                    long long nkeys, long long nplanes, long long ntab, bool planes, const int16_t* idx2,
                    const double* vt, DiamScratch& s, DiamOut* out, DiamStats* stats, cudaStream_t st, int which) {
  const rad_tuning_t& tu = tuning();
  Params p;
  p.n = n;
  p.TS = tu.tile;
  p.nplanes = nplanes;
  const long long nv = std::max<long long>(nv_cap, 2);
  p.nv_cap = nv_cap;
  p.sweep_min = (long long)kBigTiles * p.TS;  // the ROIs whose 3D problem is walked at two levels
  const long long nsorted = nv * (planes ? 4 : 1);
  // soft maps with planes: groups of vertices off the grid planes (two or
  // more vertices each), one key per group after all ROIs' keys, and a spare
  FracState fs;
  const bool frac = planes && vt != nullptr;
  long long hsize = 0;
  if (frac) {
    fs.gcap = nv / 2 + 1;
    fs.fbase = nkeys;
    hsize = 16;  // 16 keys fill one 256-byte carve unit: the counts follow the keys directly
    while (hsize < 2 * nv) hsize <<= 1;
    fs.hmask = hsize - 1;
  }
  const long long nkeys_all = nkeys + (frac ? fs.gcap + 1 : 0);
  p.max_problems = 2 * (n + nplanes + (frac ? fs.gcap : 0)) + 2;  // a problem walked at two levels takes two slots
  p.max_tiles = nsorted / p.TS + p.max_problems + 1;
  p.max_fine = nsorted / p.TS + p.max_problems + 1;
  if (s.work_cap == 0) s.work_cap = 1 << 20;
  if (s.cand_cap == 0) s.cand_cap = 1 << 20;
  p.work_cap = s.work_cap;
  p.cand_cap = s.cand_cap;
  p.refine_cap = std::max<long long>(4096, s.work_cap / 8);  // grows with the work list
  const long long ntiles = p.max_tiles + p.max_fine;

  // scratch layout (hist/offsets carry one extra entry: offs[K] = total)
  const long long K1 = nkeys_all + 1;
  const long long nparts = (K1 + kScanBlock - 1) / kScanBlock;
  size_t bytes = 0;
  auto add = [&](size_t m) { bytes += (m + 255) & ~size_t(255); };
  add(sizeof(int) * K1);             // hist
  add(sizeof(int) * K1);             // cursor
  add(sizeof(long long) * K1);       // offsets
  add(sizeof(ScanTile<1>) * nparts + 16);  // look-back state of the key scan and its ticket
  add(sizeof(float4) * nsorted);
  add(sizeof(int) * nsorted);  // vertex id of every sorted entry
  add(sizeof(Problem) * p.max_problems);
  add(sizeof(Tile) * ntiles);
  add(sizeof(int) * ntiles);    // chunk0
  add(sizeof(float4) * 2 * ntiles);
  add(sizeof(float4) * ntiles);
  add(sizeof(ProblemState) * 4 * n + sizeof(unsigned long long) * n);  // family states, sweep slots
  add(sizeof(RefineItem) * p.refine_cap);
  add(sizeof(Counters));
  add(sizeof(WorkItem) * p.work_cap);
  add(sizeof(float) * 8 * p.work_cap);  // slice maxima (up to 8 slices per item)
  add(sizeof(int) * 8 * p.work_cap);    // slices to rescan
  add(sizeof(Cand) * p.cand_cap);
  add(sizeof(float) * std::max<long long>(ntab, 1));  // coordinate tables (masks)
  add(sizeof(Key128) * 4 * n);  // family maxima of the FP64 pair kernel
  if (frac) {
    add(sizeof(Key128) * hsize);  // hash keys, then counts: one zeroed range
    add(sizeof(int) * hsize);
    add(sizeof(int) * hsize);     // group of a slot
    add(sizeof(int) * nv);        // slot of a vertex
    add(sizeof(int) * fs.gcap);   // (ROI, axis) of a group
  }
  RAD_TRY(s.misc.reserve(bytes));
  char* cur = s.misc.as<char>();
  int* hist = carve<int>(cur, K1);
  int* cursor = carve<int>(cur, K1);
  long long* offs = carve<long long>(cur, K1);
  char* scan_state = carve<char>(cur, sizeof(ScanTile<1>) * nparts + 16);
  ScanTile<1>* stiles = reinterpret_cast<ScanTile<1>*>(scan_state);
  unsigned int* stick = reinterpret_cast<unsigned int*>(scan_state + sizeof(ScanTile<1>) * nparts);
  float4* sorted = carve<float4>(cur, nsorted);
  int* ids = carve<int>(cur, nsorted);
  Problem* probs = carve<Problem>(cur, p.max_problems);
  Tile* tiles = carve<Tile>(cur, ntiles);
  int* chunk0 = carve<int>(cur, ntiles);
  float4* box = carve<float4>(cur, 2 * ntiles);
  float4* rep = carve<float4>(cur, ntiles);
  const size_t fam_bytes = sizeof(ProblemState) * 4 * n + sizeof(unsigned long long) * n;
  char* fam_state = carve<char>(cur, fam_bytes);
  ProblemState* ps = reinterpret_cast<ProblemState*>(fam_state);
  unsigned long long* sweep = reinterpret_cast<unsigned long long*>(fam_state + sizeof(ProblemState) * 4 * n);
  RefineItem* refine = carve<RefineItem>(cur, p.refine_cap);
  Counters* cnt = carve<Counters>(cur, 1);
  WorkItem* work = carve<WorkItem>(cur, p.work_cap);
  float* slicemax = carve<float>(cur, 8 * p.work_cap);
  int* hits = carve<int>(cur, 8 * p.work_cap);
  Cand* cand = carve<Cand>(cur, p.cand_cap);
  float* ctab = carve<float>(cur, std::max<long long>(ntab, 1));
  Key128* keys = carve<Key128>(cur, 4 * n);
  if (frac) {
    fs.hkey = carve<Key128>(cur, hsize);
    fs.hcnt = carve<int>(cur, hsize);
    fs.hgid = carve<int>(cur, hsize);
    fs.vslot = carve<int>(cur, nv);
    fs.gra = carve<int>(cur, fs.gcap);
  }

  const int sms = num_sms();
  ZeroSet zs{};
  zero_add(zs, hist, sizeof(int) * K1);      // carved in 256-byte units: whole words stay inside
  zero_add(zs, cursor, sizeof(int) * K1);
  zero_add(zs, cnt, sizeof(Counters));
  zero_add(zs, scan_state, sizeof(ScanTile<1>) * nparts + 16);
  zero_add(zs, stats, sizeof(DiamStats));
  zero_add(zs, fam_state, fam_bytes);  // F = T = 0 for every family; sweep slots
  zero_add(zs, keys, sizeof(Key128) * 4 * n);  // family keys of the FP64 confirmation (or FP64 pair mode)
  if (frac) zero_add(zs, fs.hkey, (sizeof(Key128) + sizeof(int)) * hsize);  // keys and counts (adjacent)
  if (which & 1) {
    // on its own (a graph branch beside the mesh) it needs few CTAs: a few MB zeroed
    const long long init_ctas = (std::max(K1, ntab) + 255) / 256;
    RAD_LAUNCH("diam_init", k_diam_init,
               wave_grid(k_diam_init, 256, which == 1 ? std::min<long long>(init_ctas, sms) : init_ctas), 256, 0, st,
               out, n, zs, rd, ctab, planes ? ntab : 0);
  }
  if (!(which & 2)) return RAD_OK;
  if (frac) {
    RAD_LAUNCH("diam_frac_insert", k_frac_insert, wave_grid(k_frac_insert, 256, (nv + 255) / 256), 256, 0, st, idx2,
               vt, nv_dev, ro, p, fs, cnt);
    RAD_LAUNCH("diam_frac_assign", k_frac_assign, wave_grid(k_frac_assign, 256, (hsize + 255) / 256), 256, 0, st, fs,
               cnt);
  }
  RAD_LAUNCH("diam_hist", k_hist, wave_grid(k_hist, 256, (nv + 255) / 256), 256, 0, st, idx2, vt, nv_dev, rd, ro, p,
             ctab, hist, sweep, ps, fs);
  RAD_LAUNCH("diam_scan", k_xscan, (int)nparts, kScanThreads, 0, st, hist, K1, (int)nparts, offs, stiles, stick,
             &cnt->status);
  RAD_LAUNCH("diam_scatter", k_scatter, wave_grid(k_scatter, 256, (nv + 255) / 256), 256, 0, st, idx2, vt, nv_dev, rd,
             ro, p, offs, cursor, ctab, sorted, ids, sweep, ps, fs);
  RAD_LAUNCH("diam_setup", k_setup, wave_grid(k_setup, 256, (n + nplanes + (frac ? fs.gcap : 0) + 255) / 256 + 1), 256,
             0, st, rd, p, offs, probs, chunk0, cnt, fs);
  // grids no larger than the host-side bounds of their work (small ROIs then
  // launch a few blocks instead of a full wave): one warp per tile; (tile row,
  // chunk) items are at most tiles x chunks per row; coarse pairs exist only
  // when one problem can reach kBigTiles tiles
  const long long tile_blocks = (p.max_tiles + p.max_fine + 7) / 8;
  const long long walk_items = p.max_tiles * ((p.max_tiles + kChunk - 1) / kChunk);
  const long long walk_blocks = (walk_items + 7) / 8;
  const bool can_coarse = nsorted >= (long long)kBigTiles * p.TS;
  RAD_LAUNCH("diam_tile_box", k_tile_box, wave_grid(k_tile_box, 256, tile_blocks), 256, 0, st, sorted, probs, p, cnt,
             tiles, chunk0, box, rep);
  RAD_LAUNCH("diam_seed", k_seed, wave_grid(k_seed, 256, walk_blocks), 256, 0, st, sorted, rep, p, tiles, chunk0, cnt, ps,
             rd, box);
  RAD_LAUNCH("diam_cull", k_cull, wave_grid(k_cull, 256, walk_blocks), 256, 0, st, tiles, box, p, chunk0, cnt, ps, work,
             refine);
  RAD_LAUNCH("diam_refine", k_refine, wave_grid(k_refine, 256, can_coarse ? std::max<long long>(1, p.refine_cap / 8) : 1),
             256, 0, st,
             tiles, box, p, cnt, ps, refine, work);
  const int ctas = sms * tu.ctas_per_sm;
  if (s.fp64_pairs) {  // every surviving pair in FP64: no filter, no candidates
    if (tu.tile == 64) {
      RAD_LAUNCH("diam_pairs_fp64", k_pairs64<64>, wave_grid(k_pairs64<64>, kP64Threads, 1LL << 30), kP64Threads, 0, st,
                 ids, idx2, vt, work, p, rd, ro, cnt, ps, keys);
    } else if (tu.tile == 128) {
      RAD_LAUNCH("diam_pairs_fp64", k_pairs64<128>, wave_grid(k_pairs64<128>, kP64Threads, 1LL << 30), kP64Threads, 0,
                 st, ids, idx2, vt, work, p, rd, ro, cnt, ps, keys);
    } else {
      RAD_LAUNCH("diam_pairs_fp64", k_pairs64<256>, wave_grid(k_pairs64<256>, kP64Threads, 1LL << 30), kP64Threads, 0,
                 st, ids, idx2, vt, work, p, rd, ro, cnt, ps, keys);
    }
    RAD_LAUNCH("diam_keys_out", k_keys_out, std::max(1, std::min(sms, (4 * n + 255) / 256)), 256, 0, st, keys, n, out);
    RAD_LAUNCH("diam_stats", k_stats, 1, 32, 0, st, cnt, stats);
    return RAD_OK;
  }
  if (tu.tile == 64) {
    if (tu.threads == 64) RAD_TRY((launch_pairs<64, 64>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
    else RAD_TRY((launch_pairs<64, 128>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
  } else if (tu.tile == 128) {
    if (tu.threads == 64) RAD_TRY((launch_pairs<128, 64>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
    else if (tu.threads == 128) RAD_TRY((launch_pairs<128, 128>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
    else RAD_TRY((launch_pairs<128, 256>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
  } else {
    if (tu.threads == 64) RAD_TRY((launch_pairs<256, 64>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
    else RAD_TRY((launch_pairs<256, 128>(sorted, work, p, rd, cnt, ps, slicemax, hits, cand, ctas, st)));
  }
  RAD_LAUNCH("diam_confirm", k_confirm, sms, 256, 0, st, ids, idx2, vt, p, rd, ro, cnt, cand, keys, out, stats);
  return RAD_OK;
}

// ---- plain FP64 all-pairs (comparison kernel) ------------------------------------

namespace {

constexpr int kPlainTile = 256;

__device__ __forceinline__ void take_best(BestD& b, double d2, int i, int j) {
  if (better(d2, i, j, b)) { b.d2 = d2; b.i = i; b.j = j; }
}

// Persistent grid over the upper-triangular tile pairs; each CTA keeps its
// running (d2, i, j) for 3D, Slice, Column, Row and writes them to scratch.
__global__ void __launch_bounds__(kPlainTile) k_plain(const int16_t* idx2, const double* vt,
                                                      int n, double sx, double sy, double sz,
                                                      BestD* part) {
  pdl_enter();
  __shared__ double su[3][kPlainTile];
  __shared__ int sq[3][kPlainTile];
  __shared__ BestD sred[4][kPlainTile / 32];
  const int nt = (n + kPlainTile - 1) / kPlainTile;
  const long long npairs = (long long)nt * (nt + 1) / 2;
  BestD b[4];
  for (int q = 0; q < 4; ++q) { b[q].d2 = 0.0; b[q].i = -1; b[q].j = -1; }
  for (long long l = blockIdx.x; l < npairs; l += gridDim.x) {
    long long tb = (long long)((sqrt(8.0 * (double)l + 1.0) - 1.0) * 0.5);
    while (tb * (tb + 1) / 2 > l) --tb;
    while ((tb + 1) * (tb + 2) / 2 <= l) ++tb;
    const long long ta = l - tb * (tb + 1) / 2;
    const int jb = (int)tb * kPlainTile;
    __syncthreads();
    {
      const int j = jb + threadIdx.x;
      if (j < n) {
        double u[3];
        vertex_u(idx2, vt, j, u);
        for (int k = 0; k < 3; ++k) { su[k][threadIdx.x] = u[k]; sq[k][threadIdx.x] = idx2[3 * j + k]; }
      }
    }
    __syncthreads();
    const int i = (int)ta * kPlainTile + threadIdx.x;
    if (i < n) {
      double ui[3];
      vertex_u(idx2, vt, i, ui);
      const int qi0 = idx2[3 * i], qi1 = idx2[3 * i + 1], qi2 = idx2[3 * i + 2];
      const int jend = min(kPlainTile, n - jb);
      for (int jj = 0; jj < jend; ++jj) {
        const int j = jb + jj;
        if (j <= i) continue;
        const double d2 = pin_d2(ui[0], ui[1], ui[2], su[0][jj], su[1][jj], su[2][jj], sx, sy, sz);
        take_best(b[0], d2, i, j);
        if (vt == nullptr) {
          if (qi2 == sq[2][jj]) take_best(b[1], d2, i, j);
          if (qi1 == sq[1][jj]) take_best(b[2], d2, i, j);
          if (qi0 == sq[0][jj]) take_best(b[3], d2, i, j);
        } else {
          if (ui[2] == su[2][jj]) take_best(b[1], d2, i, j);
          if (ui[1] == su[1][jj]) take_best(b[2], d2, i, j);
          if (ui[0] == su[0][jj]) take_best(b[3], d2, i, j);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      BestD o;
      o.d2 = __shfl_xor_sync(0xffffffffu, b[q].d2, off);
      o.i = __shfl_xor_sync(0xffffffffu, b[q].i, off);
      o.j = __shfl_xor_sync(0xffffffffu, b[q].j, off);
      if (better(o.d2, o.i, o.j, b[q])) b[q] = o;
    }
    if (lane == 0) sred[q][wid] = b[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    BestD r = sred[q][0];
    for (int w = 1; w < kPlainTile / 32; ++w)
      if (better(sred[q][w].d2, sred[q][w].i, sred[q][w].j, r)) r = sred[q][w];
    part[4 * blockIdx.x + q] = r;
  }
}

__global__ void k_plain_final(const BestD* part, int nparts, DiamResult* out) {
  pdl_enter();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    BestD r;
    r.d2 = 0.0; r.i = -1; r.j = -1;
    for (int b = 0; b < nparts; ++b)
      if (better(part[4 * b + q].d2, part[4 * b + q].i, part[4 * b + q].j, r)) r = part[4 * b + q];
    out->d2[q] = r.i >= 0 ? r.d2 : 0.0;
    out->i[q] = r.i;
    out->j[q] = r.j;
  }
}

}  // namespace

rad_status diam_plain_fp64(const int16_t* idx2, const double* vt, long long nv, const MeshDims& d, const double sp[3],
                           DiamScratch& s, DiamResult* out_dev, cudaStream_t st) {
  (void)d;
  const int ctas = num_sms() * 4;
  RAD_TRY(s.plain_part.reserve(sizeof(BestD) * 4 * ctas));
  RAD_LAUNCH("plain_fp64_pairs", k_plain, ctas, kPlainTile, 0, st, idx2, vt, (int)nv, sp[0], sp[1], sp[2],
             s.plain_part.as<BestD>());
  RAD_LAUNCH("plain_fp64_final", k_plain_final, 1, 32, 0, st, s.plain_part.as<BestD>(), ctas, out_dev);
  return RAD_OK;
}

}  // namespace rad
