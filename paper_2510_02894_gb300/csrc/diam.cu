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
//      vertex id).  The 3D problem is the whole cell-sorted range; every plane
//      with two or more vertices is its own problem.
//   2. Each problem is cut into tiles of TS vertices; a tile gets its
//      bounding box and 14 directional extremes.  The pairs of each
//      problem's extremes seed its running maximum F.
//   3. Tile pairs whose farthest-corner bound cannot reach the threshold
//      T(F) are culled; the rest form a device work list.
//   4. A persistent kernel evaluates the surviving tile pairs in FP32 from
//      shared memory (6 FP32 operations per pair, warp max, one atomic max
//      per tile pair on F), re-culling each item against the current F.
//   5. Pairs with f >= T(F) become candidates and are re-evaluated in FP64
//      with the pinned formula; max d2, then the smallest (i, j).
//
// FP32 error bound (per pair, binary or soft; u = 2^-24, positions a relative
// to the grid centre, R = the grid's half extent in mm):
//   P_k = fl32(a_k),  dx = fl(P_i - P_j),  f = fma(dz,dz, fma(dy,dy, dx*dx))
//   |f - d2| <= 5.1u d2 + 4.1u |R| sqrt(d2) + 4.1u^2 |R|^2.
// T(F) inverts this bound (with every coefficient doubled), so every pair
// attaining the FP64 maximum has f >= T(F) for any F not above the largest
// f; the culling bound uses the same monotone FP32 operations on box
// distances, so it bounds f from above without any epsilon.
#include <float.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "rad_internal.cuh"

namespace rad {

namespace {


struct Problem {
  int axis;  // -1: 3D, 0: Row (equal x), 1: Column (equal y), 2: Slice (equal z)
  int beg, len;
  int tile_beg;  // first tile
  int roi;
  int pad;
};

struct Tile {
  int problem, beg, len, tile_end;  // tile_end: one past the problem's last tile
};

struct WorkItem {
  int problem, ta, tb, roi;
};

struct Cand {
  int ea, eb, problem, roi;
};

struct ProblemState {
  unsigned int F;  // float bits of the running FP32 maximum
  unsigned int T;  // float bits of T(F), raised with F
  unsigned long long best_d2;    // FP64 bits of the confirmed maximum
  unsigned long long best_pair;  // (i << 32) | j, smallest among the maxima
};

struct Counters {
  int n_problems;
  int n_tiles;
  long long n_pairs;
  long long n_work;
  long long n_cand;
  int ticket;
  int ticket2;
  unsigned int status;
  int pad;
  unsigned long long items_evaluated, pairs_evaluated;
  long long n_work2;  // items re-evaluated for candidates
  unsigned int done;  // last-block ticket
  unsigned int pad2;
};

// Batch-wide parameters of one run.
struct Params {
  int n;              // ROIs
  int TS;
  long long nplanes;  // planes of all ROIs
  long long work_cap, cand_cap, max_problems, max_tiles;
  long long nv_cap;   // vertex pool capacity: device counts are clamped to it
};

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

// Warp-aggregated: lanes with equal keys (consecutive vertices share cells and
// planes) make one atomic.
__global__ void k_hist(const int16_t* __restrict__ idx2, const long long* __restrict__ nv_dev,
                       const RoiDiam* __restrict__ rd, const RoiOut* __restrict__ ro, Params p,
                       int* __restrict__ hist) {
  const long long n = min(*nv_dev, p.nv_cap);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; v0 < n; v0 += stride) {
    const long long v = v0 + lane;
    int q[3] = {0, 0, 0};
    int roi = 0;
    if (v < n) {
      vertex_q(idx2, v, q);
      roi = p.n == 1 ? 0 : roi_of_vertex(ro, p.n, v);
    }
    const RoiDiam& r = rd[roi];
    for (int k = 0; k < 4; ++k) {
      const bool use = v < n && (k == 0 || r.planes);
      const long long key = use ? key_of(r, q, k) : -1;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[key], __popc(peers));
    }
  }
}

__device__ __forceinline__ long long key_offset(const long long* offs, const long long* parts, long long key);

__global__ void k_scatter(const int16_t* __restrict__ idx2, const double* __restrict__ vt,
                          const long long* __restrict__ nv_dev, const RoiDiam* __restrict__ rd,
                          const RoiOut* __restrict__ ro, Params p, const long long* __restrict__ offs,
                          const long long* __restrict__ parts, int* __restrict__ cursor,
                          float4* __restrict__ sorted) {
  const long long n = min(*nv_dev, p.nv_cap);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; v0 < n; v0 += stride) {
    const long long v = v0 + lane;
    int q[3] = {0, 0, 0};
    int roi = 0;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v < n) {
      vertex_q(idx2, v, q);
      roi = p.n == 1 ? 0 : roi_of_vertex(ro, p.n, v);
      const RoiDiam& r = rd[roi];
      double u[3];
      vertex_u(idx2, vt, v, u);
      e = make_float4(__double2float_rn((u[0] - r.cx) * r.sx), __double2float_rn((u[1] - r.cy) * r.sy),
                      __double2float_rn((u[2] - r.cz) * r.sz), __int_as_float((int)v));
    }
    const RoiDiam& r = rd[roi];
    for (int k = 0; k < 4; ++k) {
      const bool use = v < n && (k == 0 || r.planes);
      const long long key = use ? key_of(r, q, k) : -1;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      int base = 0;
      if (key >= 0 && lane == leader) base = atomicAdd(&cursor[key], __popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (key >= 0) sorted[key_offset(offs, parts, key) + base + __popc(peers & ((1u << lane) - 1u))] = e;
    }
  }
}

// Generic exclusive scan of int counts to long long offsets (3 kernels).
constexpr int kScanBlock = 1024;
__global__ void k_xscan_part(const int* __restrict__ in, long long n, long long* __restrict__ out,
                             long long* __restrict__ part) {
  __shared__ long long ws[32];
  const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
  long long v = i < n ? in[i] : 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc = v;
  for (int off = 1; off < 32; off <<= 1) {
    const long long o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  long long wb = 0, tot = 0;
  for (int k = 0; k < kScanBlock / 32; ++k) {
    if (k < wid) wb += ws[k];
    tot += ws[k];
  }
  if (i < n) out[i] = wb + inc - v;
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_xscan_top(long long* __restrict__ part, int nparts) {
  __shared__ long long ws[32];
  long long carry = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < nparts; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const long long v = i < nparts ? part[i] : 0;
    long long inc = v;
    for (int off = 1; off < 32; off <<= 1) {
      const long long o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    long long wb = 0, tot = 0;
    for (int k = 0; k < nw; ++k) {
      if (k < wid) wb += ws[k];
      tot += ws[k];
    }
    if (i < nparts) part[i] = carry + wb + inc - v;
    carry += tot;
    __syncthreads();
  }
}

// Offset of a key: block-local exclusive prefix + the scanned block total.
__device__ __forceinline__ long long key_offset(const long long* offs, const long long* parts, long long key) {
  return offs[key] + parts[key / kScanBlock];
}

// ---- 2. problems and tiles --------------------------------------------------------
// One warp per candidate problem: the 3D problem of every ROI (items 0..n-1)
// and every plane of every ROI (items n..).  A problem with >= 2 vertices
// takes a slot and a contiguous run of tiles with atomics (the order of
// problems does not affect any result), resets its state and writes its
// tiles.
__device__ __forceinline__ int roi_of_plane(const RoiDiam* rd, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rd[mid].plane0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_setup(const RoiDiam* __restrict__ rd, Params p, const long long* __restrict__ offs,
                        const long long* __restrict__ parts, Problem* __restrict__ probs, Tile* __restrict__ tiles,
                        ProblemState* __restrict__ ps, Counters* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long items = p.n + p.nplanes;
  for (long long it = warp; it < items; it += nwarps) {
    int roi, axis;
    long long k0, k1;
    if (it < p.n) {
      roi = (int)it;
      const RoiDiam& r = rd[roi];
      axis = -1;
      k0 = r.key0;
      k1 = r.key0 + r.C3;
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
    const long long beg = key_offset(offs, parts, k0);
    const long long len = key_offset(offs, parts, k1) - beg;
    if (len < 2) continue;  // warp-uniform
    const int nt = (int)((len + p.TS - 1) / p.TS);
    int slot = 0, tb = 0;
    if (lane == 0) {
      slot = atomicAdd(&cnt->n_problems, 1);
      tb = atomicAdd(&cnt->n_tiles, nt);
      atomicAdd((unsigned long long*)&cnt->n_pairs, (unsigned long long)nt * (nt + 1) / 2);
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    tb = __shfl_sync(0xffffffffu, tb, 0);
    if (slot >= p.max_problems || (long long)tb + nt > p.max_tiles) {
      if (lane == 0) atomicOr(&cnt->status, DEV_ERR_PROBCAP);
      continue;
    }
    if (lane == 0) {
      Problem q;
      q.axis = axis; q.beg = (int)beg; q.len = (int)len; q.tile_beg = tb; q.roi = roi; q.pad = 0;
      probs[slot] = q;
      ProblemState z;
      z.F = 0u; z.T = 0u; z.best_d2 = 0ull; z.best_pair = ~0ull;
      ps[slot] = z;
    }
    for (int t = lane; t < nt; t += 32) {
      Tile tl;
      tl.problem = slot;
      tl.beg = (int)beg + t * p.TS;
      tl.len = min(p.TS, (int)len - t * p.TS);
      tl.tile_end = tb + nt;
      tiles[tb + t] = tl;
    }
  }
}

// One warp per tile: bounding box of its FP32 positions.
__global__ void k_tile_box(const float4* __restrict__ sorted, const Tile* __restrict__ tiles, Params p,
                           const Counters* __restrict__ cnt, float4* __restrict__ box, float4* __restrict__ rep) {
  const int nt = (int)min((long long)cnt->n_tiles, p.max_tiles);
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long ti = warp; ti < nt; ti += nwarps) {
    const Tile tl = tiles[ti];
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = lane; i < tl.len; i += 32) {
      const float4 v = sorted[tl.beg + i];
      lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
      hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
    }
    for (int off = 16; off > 0; off >>= 1)
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
        hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
      }
    if (lane == 0) {
      box[2 * ti] = make_float4(lo[0], lo[1], lo[2], 0.f);
      box[2 * ti + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
      rep[ti] = sorted[tl.beg];
    }
  }
}

// Seed: one warp per tile row a.  The pairs of tile representatives (first
// vertex of each tile) of one problem, plus each tile's first-last pair, are
// actual vertex pairs, so their largest f is a valid starting F.
__global__ void k_seed_rows(const float4* __restrict__ sorted, const float4* __restrict__ rep, Params p,
                            const RoiDiam* __restrict__ rd, const Problem* __restrict__ probs,
                            const Tile* __restrict__ tiles, Counters* __restrict__ cnt,
                            ProblemState* __restrict__ ps) {
  const int nt = (int)min((long long)cnt->n_tiles, p.max_tiles);
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long a = warp; a < nt; a += nwarps) {
    const Tile ta = tiles[a];
    const float4 ra = rep[a];
    float best = lane == 0 ? pair_f(ra, sorted[ta.beg + ta.len - 1]) : 0.0f;
    for (long long b = a + 1 + lane; b < ta.tile_end; b += 32) best = fmaxf(best, pair_f(ra, rep[b]));
    for (int off = 16; off > 0; off >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
    if (lane == 0 && best > 0.0f) atomicMax(&ps[ta.problem].F, __float_as_uint(best));
  }
  // the last block turns every seeded F into its threshold T(F) (FP64 math
  // once per problem instead of once per tile row)
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&cnt->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const int np = (int)min((long long)cnt->n_problems, p.max_problems);
    for (int i = threadIdx.x; i < np; i += blockDim.x)
      ps[i].T = __float_as_uint(threshold(__uint_as_float(__ldcg(&ps[i].F)), rd[probs[i].roi]));
    __syncthreads();
    if (threadIdx.x == 0) cnt->done = 0;
  }
}

// ---- 3. culling -------------------------------------------------------------------
// One warp per tile row a: every tile pair (a, b >= a) of the same problem
// whose box bound reaches T(F) goes to the work list.
__global__ void k_cull_rows(const Tile* __restrict__ tiles, const float4* __restrict__ box, Params p,
                            const Problem* __restrict__ probs, Counters* __restrict__ cnt,
                            ProblemState* __restrict__ ps, WorkItem* __restrict__ work) {
  const int nt = (int)min((long long)cnt->n_tiles, p.max_tiles);
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long a = warp; a < nt; a += nwarps) {
    const Tile ta = tiles[a];
    const float T = __uint_as_float(ps[ta.problem].T);
    const int roi = probs[ta.problem].roi;
    const float4 alo = box[2 * a], ahi = box[2 * a + 1];
    for (long long b0 = a; b0 < ta.tile_end; b0 += 32) {
      const long long b = b0 + lane;
      bool keep = false;
      if (b < ta.tile_end) keep = box_ub(alo, ahi, box[2 * b], box[2 * b + 1]) >= T;
      const unsigned int m = __ballot_sync(0xffffffffu, keep);
      if (!m) continue;
      long long base = 0;
      if (lane == 0) base = atomicAdd((unsigned long long*)&cnt->n_work, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) {
        const long long slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < p.work_cap) {
          WorkItem w;
          w.problem = ta.problem; w.ta = (int)a; w.tb = (int)b; w.roi = roi;
          work[slot] = w;
        } else {
          atomicOr(&cnt->status, DEV_ERR_WORKCAP);
        }
      }
    }
  }
}

// Items whose FP32 maximum reaches the final threshold of their problem are
// re-evaluated for candidates; list them compactly.
__global__ void k_compact_items(const WorkItem* __restrict__ work, const float* __restrict__ itemmax, Params p,
                                Counters* __restrict__ cnt, const ProblemState* __restrict__ ps,
                                int* __restrict__ work2) {
  const long long nwork = min(cnt->n_work, p.work_cap);
  const int lane = threadIdx.x & 31;
  for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < nwork; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    bool keep = false;
    if (i < nwork) keep = itemmax[i] >= __uint_as_float(ps[work[i].problem].T);
    const unsigned int m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    long long base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long*)&cnt->n_work2, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) work2[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
  }
}

// ---- 4./5. pair kernels ------------------------------------------------------------

// Evaluates one tile pair from shared memory.  NT threads; lane l of every
// warp holds the A entries l, l + 32, ...; warp w scans its slice of B.
template <int TS, int NT, bool CAND>
__device__ __forceinline__ float eval_pair_tile(const float4* __restrict__ sorted, const Tile& A, const Tile& B,
                                                float4* sB, float T, int problem, int roi, Cand* cand, Counters* cnt,
                                                long long cand_cap) {
  constexpr int RA = TS / 32;
  constexpr int NWARP = NT / 32;
  constexpr int BSL = TS / NWARP;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < TS; i += NT) sB[i] = i < B.len ? sorted[B.beg + i] : sorted[B.beg];
  float4 a[RA];
  for (int r = 0; r < RA; ++r) {
    const int ia = lane + 32 * r;
    a[r] = sorted[A.beg + min(ia, A.len - 1)];
  }
  __syncthreads();
  float mx[RA];
  for (int r = 0; r < RA; ++r) mx[r] = 0.0f;
  const int jb = wid * BSL;
  const int je = min(jb + BSL, B.len);
  if (!CAND) {
#pragma unroll 4
    for (int j = jb; j < je; ++j) {
      const float4 b = sB[j];
#pragma unroll
      for (int r = 0; r < RA; ++r) mx[r] = fmaxf(mx[r], pair_f(a[r], b));
    }
  } else {
    for (int j = jb; j < je; ++j) {
      const float4 b = sB[j];
      for (int r = 0; r < RA; ++r) {
        const int ia = lane + 32 * r;
        if (ia >= A.len) continue;
        const int ea = A.beg + ia, eb = B.beg + j;
        if (A.beg == B.beg && ea >= eb) continue;  // same tile: each unordered pair once
        const float f = pair_f(a[r], b);
        if (f >= T) {
          const long long slot = atomicAdd((unsigned long long*)&cnt->n_cand, 1ull);
          if (slot < cand_cap) {
            Cand c;
            c.ea = ea; c.eb = eb; c.problem = problem; c.roi = roi;
            cand[slot] = c;
          } else {
            atomicOr(&cnt->status, DEV_ERR_CANDCAP);
          }
        }
      }
    }
  }
  float m = 0.0f;
  for (int r = 0; r < RA; ++r)
    if (lane + 32 * r < A.len) m = fmaxf(m, mx[r]);
  return m;
}

template <int TS, int NT>
__global__ void __launch_bounds__(NT) k_pairs_max(const float4* __restrict__ sorted, const Tile* __restrict__ tiles,
                                                  const float4* __restrict__ box, const WorkItem* __restrict__ work,
                                                  Params p, const RoiDiam* __restrict__ rd,
                                                  Counters* __restrict__ cnt, ProblemState* __restrict__ ps,
                                                  float* __restrict__ itemmax) {
  __shared__ float4 sB[TS];
  __shared__ float sred[NT / 32];
  const long long nwork = min(cnt->n_work, p.work_cap);
  unsigned long long n_items = 0, n_pairs = 0;
  for (long long it = blockIdx.x; it < nwork; it += gridDim.x) {
    const WorkItem w = work[it];
    // re-cull against the problem's current threshold (raised by other CTAs);
    // threads may read different values, so the decision is block-wide
    const float T = __uint_as_float(*(volatile unsigned int*)&ps[w.problem].T);
    const float ub = box_ub(box[2 * w.ta], box[2 * w.ta + 1], box[2 * w.tb], box[2 * w.tb + 1]);
    if (__syncthreads_and(ub < T)) {
      if (threadIdx.x == 0) itemmax[it] = -1.0f;
      continue;
    }
    const Tile A = tiles[w.ta], B = tiles[w.tb];
    float m = eval_pair_tile<TS, NT, false>(sorted, A, B, sB, T, w.problem, w.roi, nullptr, cnt, 0);
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float bm = sred[0];
      for (int k = 1; k < NT / 32; ++k) bm = fmaxf(bm, sred[k]);
      itemmax[it] = bm;
      const unsigned int old = atomicMax(&ps[w.problem].F, __float_as_uint(bm));
      if (__float_as_uint(bm) > old) atomicMax(&ps[w.problem].T, __float_as_uint(threshold(bm, rd[w.roi])));
      n_items++;
      n_pairs += (unsigned long long)A.len * (unsigned long long)B.len;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && n_items) {
    atomicAdd(&cnt->items_evaluated, n_items);
    atomicAdd(&cnt->pairs_evaluated, n_pairs);
  }
}

template <int TS, int NT>
__global__ void __launch_bounds__(NT) k_pairs_cand(const float4* __restrict__ sorted, const Tile* __restrict__ tiles,
                                                   const WorkItem* __restrict__ work, const int* __restrict__ work2,
                                                   Params p, Counters* __restrict__ cnt,
                                                   const ProblemState* __restrict__ ps, Cand* __restrict__ cand) {
  __shared__ float4 sB[TS];
  const long long n2 = cnt->n_work2;
  for (long long k = blockIdx.x; k < n2; k += gridDim.x) {
    const WorkItem w = work[work2[k]];
    const float T = __uint_as_float(ps[w.problem].T);
    const Tile A = tiles[w.ta], B = tiles[w.tb];
    eval_pair_tile<TS, NT, true>(sorted, A, B, sB, T, w.problem, w.roi, cand, cnt, p.cand_cap);
    __syncthreads();
  }
}

// ---- 5. FP64 confirmation -------------------------------------------------------------

__global__ void k_confirm(const float4* __restrict__ sorted, const int16_t* __restrict__ idx2,
                          const double* __restrict__ vt, Params p, const RoiDiam* __restrict__ rd,
                          const Counters* __restrict__ cnt, const Cand* __restrict__ cand,
                          ProblemState* __restrict__ ps) {
  const long long nc = min(cnt->n_cand, p.cand_cap);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const Cand k = cand[c];
    const RoiDiam& r = rd[k.roi];
    const int i = __float_as_int(sorted[k.ea].w), j = __float_as_int(sorted[k.eb].w);
    double ui[3], uj[3];
    vertex_u(idx2, vt, i, ui);
    vertex_u(idx2, vt, j, uj);
    const double d2 = pin_d2(ui[0], ui[1], ui[2], uj[0], uj[1], uj[2], r.sx, r.sy, r.sz);
    atomicMax(&ps[k.problem].best_d2, (unsigned long long)__double_as_longlong(d2));
  }
}

// Candidates attaining their problem's maximum take the smallest (i, j)
// (ids local to the ROI).  The last block to finish then reduces the
// problems to one result per ROI and category (3D, Slice, Column, Row): first
// the largest d2, then the smallest pair among the problems attaining it.
__global__ void k_tiebreak(const float4* __restrict__ sorted, const int16_t* __restrict__ idx2,
                           const double* __restrict__ vt, Params p, const RoiDiam* __restrict__ rd,
                           const RoiOut* __restrict__ ro, Counters* __restrict__ cnt, const Cand* __restrict__ cand,
                           ProblemState* __restrict__ ps, const Problem* __restrict__ probs,
                           DiamOut* __restrict__ out, DiamStats* __restrict__ stats) {
  const long long nc = min(cnt->n_cand, p.cand_cap);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const Cand k = cand[c];
    const RoiDiam& r = rd[k.roi];
    int i = __float_as_int(sorted[k.ea].w), j = __float_as_int(sorted[k.eb].w);
    double ui[3], uj[3];
    vertex_u(idx2, vt, i, ui);
    vertex_u(idx2, vt, j, uj);
    const double d2 = pin_d2(ui[0], ui[1], ui[2], uj[0], uj[1], uj[2], r.sx, r.sy, r.sz);
    if ((unsigned long long)__double_as_longlong(d2) == __ldcg(&ps[k.problem].best_d2)) {
      const long long v0 = ro[k.roi].v0;
      i -= (int)v0;
      j -= (int)v0;
      if (i > j) { const int t = i; i = j; j = t; }
      atomicMin(&ps[k.problem].best_pair, ((unsigned long long)(unsigned int)i << 32) | (unsigned int)j);
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&cnt->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int np = (int)min((long long)cnt->n_problems, p.max_problems);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const Problem pr = probs[i];
    if (__ldcg(&ps[i].best_pair) == ~0ull) continue;
    const int q = pr.axis < 0 ? 0 : (pr.axis == 2 ? 1 : (pr.axis == 1 ? 2 : 3));
    atomicMax(&out[pr.roi].d2[q], __ldcg(&ps[i].best_d2));
  }
  __threadfence();  // phase-1 atomics of every thread visible before phase 2
  __syncthreads();
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const Problem pr = probs[i];
    const unsigned long long bp = __ldcg(&ps[i].best_pair);
    if (bp == ~0ull) continue;
    const int q = pr.axis < 0 ? 0 : (pr.axis == 2 ? 1 : (pr.axis == 1 ? 2 : 3));
    if (__ldcg(&ps[i].best_d2) == __ldcg(&out[pr.roi].d2[q])) atomicMin(&out[pr.roi].pair[q], bp);
  }
  if (threadIdx.x == 0) {
    stats->problems = cnt->n_problems;
    stats->tiles = cnt->n_tiles;
    stats->tile_pairs = cnt->n_pairs;
    stats->work_items = cnt->n_work;
    stats->items_evaluated = (long long)cnt->items_evaluated;
    stats->pairs_evaluated = (long long)cnt->pairs_evaluated;
    stats->candidates = cnt->n_cand;
    stats->status |= cnt->status;
  }
}

__global__ void k_diam_init(DiamOut* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int q = 0; q < 4; ++q) {
      out[i].d2[q] = 0ull;
      out[i].pair[q] = ~0ull;
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
rad_status launch_pairs(const float4* sorted, const Tile* tiles, const float4* box, const WorkItem* work, int* work2,
                        const Params& p, const RoiDiam* rd, Counters* cnt, ProblemState* ps, float* itemmax,
                        Cand* cand, int ctas, cudaStream_t st) {
  auto kmax = k_pairs_max<TS, NT>;
  auto kcand = k_pairs_cand<TS, NT>;
  const int sms = num_sms();
  RAD_LAUNCH("diam_pairs_fp32", kmax, ctas, NT, 0, st, sorted, tiles, box, work, p, rd, cnt, ps, itemmax);
  RAD_LAUNCH("diam_compact", k_compact_items, sms * 4, 256, 0, st, work, itemmax, p, cnt, ps, work2);
  RAD_LAUNCH("diam_pairs_cand", kcand, ctas, NT, 0, st, sorted, tiles, work, work2, p, cnt, ps, cand);
  return RAD_OK;
}

}  // namespace

// Host-side per-ROI parameters of the diameter problems.
void plan_diam(const std::vector<Roi>& rois, bool soft, std::vector<RoiDiam>& rd, long long& nkeys,
               long long& nplanes) {
  const rad_tuning_t& tu = tuning();
  rd.resize(rois.size());
  nkeys = 0;
  nplanes = 0;
  const double u = ldexp(1.0, -24);
  for (size_t i = 0; i < rois.size(); ++i) {
    const Roi& g = rois[i];
    RoiDiam& p = rd[i];
    p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
    p.planes = soft ? 0 : 1;
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
    p.alpha = 2.0 * 5.1 * u + 1e-14;
    p.beta = 2.0 * 4.1 * u * sqrt(R2);
    p.gamma = 2.0 * 4.1 * u * u * R2;
  }
}

rad_status diam_run(int n, const RoiDiam* rd, const RoiOut* ro, const long long* nv_dev, long long nv_cap,
                    long long nkeys, long long nplanes, bool planes, const int16_t* idx2, const double* vt,
                    DiamScratch& s, DiamOut* out, DiamStats* stats, cudaStream_t st) {
  const rad_tuning_t& tu = tuning();
  Params p;
  p.n = n;
  p.TS = tu.tile;
  p.nplanes = nplanes;
  const long long nv = std::max<long long>(nv_cap, 2);
  p.nv_cap = nv_cap;
  const long long nsorted = nv * (planes ? 4 : 1);
  p.max_problems = n + nplanes + 1;
  p.max_tiles = nsorted / p.TS + p.max_problems + 1;
  if (s.work_cap == 0) s.work_cap = 1 << 20;
  if (s.cand_cap == 0) s.cand_cap = 1 << 20;
  p.work_cap = s.work_cap;
  p.cand_cap = s.cand_cap;

  // scratch layout (hist/offsets carry one extra entry: offs[K] = total)
  const long long K1 = nkeys + 1;
  const long long nparts = (K1 + kScanBlock - 1) / kScanBlock;
  size_t bytes = 0;
  auto add = [&](size_t m) { bytes += (m + 255) & ~size_t(255); };
  add(sizeof(int) * K1);             // hist
  add(sizeof(int) * K1);             // cursor
  add(sizeof(long long) * K1);       // offsets
  add(sizeof(long long) * (nparts + 1));
  add(sizeof(float4) * nsorted);
  add(sizeof(Problem) * p.max_problems);
  add(sizeof(Tile) * p.max_tiles);
  add(sizeof(float4) * 2 * p.max_tiles);
  add(sizeof(float4) * p.max_tiles);
  add(sizeof(ProblemState) * p.max_problems);
  add(sizeof(Counters));
  add(sizeof(WorkItem) * p.work_cap);
  add(sizeof(float) * p.work_cap);
  add(sizeof(int) * p.work_cap);
  add(sizeof(Cand) * p.cand_cap);
  RAD_TRY(s.misc.reserve(bytes));
  char* cur = s.misc.as<char>();
  int* hist = carve<int>(cur, K1);
  int* cursor = carve<int>(cur, K1);
  long long* offs = carve<long long>(cur, K1);
  long long* parts = carve<long long>(cur, nparts + 1);
  float4* sorted = carve<float4>(cur, nsorted);
  Problem* probs = carve<Problem>(cur, p.max_problems);
  Tile* tiles = carve<Tile>(cur, p.max_tiles);
  float4* box = carve<float4>(cur, 2 * p.max_tiles);
  float4* rep = carve<float4>(cur, p.max_tiles);
  ProblemState* ps = carve<ProblemState>(cur, p.max_problems);
  Counters* cnt = carve<Counters>(cur, 1);
  WorkItem* work = carve<WorkItem>(cur, p.work_cap);
  float* itemmax = carve<float>(cur, p.work_cap);
  int* work2 = carve<int>(cur, p.work_cap);
  Cand* cand = carve<Cand>(cur, p.cand_cap);

  const int sms = num_sms();
  RAD_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * K1, st));
  RAD_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * K1, st));
  RAD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(Counters), st));
  RAD_LAUNCH("diam_init", k_diam_init, std::max(1, std::min((n + 255) / 256, sms * 4)), 256, 0, st, out, n);
  const int vblocks = (int)std::min<long long>((nv + 255) / 256, (long long)sms * 8);
  RAD_LAUNCH("diam_hist", k_hist, vblocks, 256, 0, st, idx2, nv_dev, rd, ro, p, hist);
  RAD_LAUNCH("diam_scan_part", k_xscan_part, (int)nparts, kScanBlock, 0, st, hist, K1, offs, parts);
  RAD_LAUNCH("diam_scan_top", k_xscan_top, 1, 1024, 0, st, parts, (int)nparts);
  RAD_LAUNCH("diam_scatter", k_scatter, vblocks, 256, 0, st, idx2, vt, nv_dev, rd, ro, p, offs, parts, cursor, sorted);
  RAD_LAUNCH("diam_setup", k_setup, sms * 4, 256, 0, st, rd, p, offs, parts, probs, tiles, ps, cnt);
  RAD_LAUNCH("diam_tile_box", k_tile_box, sms * 8, 256, 0, st, sorted, tiles, p, cnt, box, rep);
  RAD_LAUNCH("diam_seed", k_seed_rows, sms * 8, 256, 0, st, sorted, rep, p, rd, probs, tiles, cnt, ps);
  RAD_LAUNCH("diam_cull", k_cull_rows, sms * 8, 256, 0, st, tiles, box, p, probs, cnt, ps, work);
  const int ctas = sms * tu.ctas_per_sm;
  if (tu.tile == 64) {
    if (tu.threads == 64) RAD_TRY((launch_pairs<64, 64>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
    else RAD_TRY((launch_pairs<64, 128>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
  } else if (tu.tile == 128) {
    if (tu.threads == 64) RAD_TRY((launch_pairs<128, 64>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
    else if (tu.threads == 128) RAD_TRY((launch_pairs<128, 128>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
    else RAD_TRY((launch_pairs<128, 256>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
  } else {
    if (tu.threads == 128) RAD_TRY((launch_pairs<256, 128>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
    else RAD_TRY((launch_pairs<256, 256>(sorted, tiles, box, work, work2, p, rd, cnt, ps, itemmax, cand, ctas, st)));
  }
  RAD_LAUNCH("diam_confirm", k_confirm, sms * 4, 256, 0, st, sorted, idx2, vt, p, rd, cnt, cand, ps);
  RAD_LAUNCH("diam_tiebreak", k_tiebreak, sms * 4, 256, 0, st, sorted, idx2, vt, p, rd, ro, cnt, cand, ps, probs, out,
             stats);
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
__global__ void __launch_bounds__(kPlainTile) k_plain(const int16_t* __restrict__ idx2, const double* __restrict__ vt,
                                                      int n, double sx, double sy, double sz,
                                                      BestD* __restrict__ part) {
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

__global__ void k_plain_final(const BestD* __restrict__ part, int nparts, DiamResult* __restrict__ out) {
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
