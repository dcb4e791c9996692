// Marching cubes on padded masks (paper Sec. 2, "Marching cubes fused
// parallel kernels"): every cube of the implicitly zero-padded grid is tested
// against the iso level, crossing edges become vertices, the cube's case
// selects its polygons, and the mesh volume and surface area are summed.
//
// Every kernel covers a whole batch of regions of interest (ROIs) in one
// launch: the rows, bitset words and outputs of all ROIs are concatenated and
// each item finds its ROI in a small device table (binary search over start
// offsets).  A single mask is the one-ROI case.
//
// GB300 layout of the pass:
//   k_pack   each mask is read once, coalesced and vectorised (16-byte loads),
//            and packed to one bit per voxel (32 voxels per word) with zero
//            rows around it; the packed grid is 1/8 of the input and stays in
//            L2 for the passes below.
//   k_count  one group of lanes per x-row (y, z), two or four words per
//            lane: crossing-edge bits by XOR of neighbouring rows, counted
//            with popc; active cubes by OR/AND of the four rows of a cube
//            row; per-row vertex, triangle, voxel and active-cube counts,
//            row-local word prefixes (written only for words with surface)
//            and the list of words with surface.
//   k_scan_rows  single-pass exclusive scan of the row counts over the whole
//            batch (decoupled look-back, bounded waits): vertex and triangle
//            ids follow the canonical (z, y, x, axis) order inside each ROI,
//            ROIs one after the other.
//   k_emit   masks: warps take 32 listed words at a time; a word's vertices
//            get ids = row base + word prefix + popc rank, its active cubes
//            their twelve edge ids and triangles (a per-case table), the
//            exact int64 volume in half-voxel units
//            (6V = det(diag(s/2)) * sum A.(B x C)) and a per-ROI, per-case
//            histogram from which k_mask_totals takes the area, so both are
//            deterministic.
//   k_rows, k_cubes  soft maps (one ROI): per row its interpolated vertices
//            and a compact list of active cubes, then one thread per cube for
//            its triangles and FP64 volume and area, summed in a fixed order.
#include <array>
#include <map>
#include <mutex>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "mc_tables.inc"
#include "rad_internal.cuh"

namespace rad {

namespace {

// Eigenvalues (descending) of a symmetric 3x3 matrix by cyclic Jacobi
// rotations in FP64: each rotation zeroes one off-diagonal element, and the
// sweeps stop once the off-diagonal part is negligible against the diagonal.
// (A closed form through the characteristic cubic loses about half the digits
// of a nearly repeated eigenvalue, which the square roots of the axis lengths
// then expose; rotations keep every eigenvalue within a few ulps of |A|.)
// One division, one square root and one reciprocal square root per rotation.
__device__ void sym3_eigenvalues(double a[3][3], double lam[3]) {
  for (int sweep = 0; sweep < 16; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double diag = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-34 * diag) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        // t = tan of the rotation angle, the smaller root of t^2 + 2 theta t - 1 = 0
        const double theta = 0.5 * (a[q][q] - a[p][p]);
        const double h = sqrt(theta * theta + apq * apq);
        const double t = apq / (fabs(theta) + h) * (theta >= 0.0 ? 1.0 : -1.0);
        const double c = rsqrt(t * t + 1.0), s = t * c;
        a[p][p] -= t * apq;
        a[q][q] += t * apq;
        a[p][q] = a[q][p] = 0.0;
        const int r = 3 - p - q;
        const double arp = a[r][p], arq = a[r][q];
        a[r][p] = a[p][r] = c * arp - s * arq;
        a[r][q] = a[q][r] = s * arp + c * arq;
      }
  }
  lam[0] = a[0][0]; lam[1] = a[1][1]; lam[2] = a[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[j] > lam[i]) { const double t = lam[i]; lam[i] = lam[j]; lam[j] = t; }
}

// Closed-form Shape features into d[0..4] (Sphericity, SurfaceVolumeRatio,
// Compactness1, Compactness2, SphericalDisproportion) from the mesh volume V
// and area A; a zero denominator gives 0.
__device__ void closed_form_features(double V, double A, double* d) {
  const double pi = 3.14159265358979323846;
  const double k = cbrt(36.0 * pi * V * V);
  d[0] = A > 0.0 ? k / A : 0.0;
  d[1] = V > 0.0 ? A / V : 0.0;
  d[2] = A > 0.0 ? V / (sqrt(pi) * A * sqrt(A)) : 0.0;
  d[3] = A > 0.0 ? 36.0 * pi * V * V / (A * A * A) : 0.0;
  d[4] = k > 0.0 ? A / k : 0.0;
}

// Principal axes into d[5..9] (Major/Minor/LeastAxisLength, Elongation,
// Flatness) from the eigenvalues of the inside voxels' coordinate covariance
// (1/N normalisation).  The covariance numerators N sum(ab) - sum(a) sum(b)
// are formed exactly in 128-bit integers from the exact moments, so each
// entry is rounded once.  Eigenvalues below 0 (rounding) count as 0; with a
// zero major eigenvalue the ratios are 0.
__device__ void principal_axes(long long N, const unsigned long long* mom, double sx, double sy, double sz,
                               double* d) {
  double lam[3] = {0.0, 0.0, 0.0};
  if (N > 0) {
    const double sp[3] = {sx, sy, sz};
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};  // xx yy zz xy xz yz
    double c[3][3];
    for (int e = 0; e < 6; ++e) {
      const __int128 num = (__int128)N * (__int128)mom[3 + e] - (__int128)mom[ia[e]] * (__int128)mom[ib[e]];
      const double v = (double)num / ((double)N * (double)N) * sp[ia[e]] * sp[ib[e]];
      c[ia[e]][ib[e]] = c[ib[e]][ia[e]] = v;
    }
    sym3_eigenvalues(c, lam);
  }
  for (int k = 0; k < 3; ++k) lam[k] = lam[k] > 0.0 ? lam[k] : 0.0;
  d[5] = 4.0 * sqrt(lam[0]);
  d[6] = 4.0 * sqrt(lam[1]);
  d[7] = 4.0 * sqrt(lam[2]);
  d[8] = lam[0] > 0.0 ? sqrt(lam[1] / lam[0]) : 0.0;
  d[9] = lam[0] > 0.0 ? sqrt(lam[2] / lam[0]) : 0.0;
}

constexpr int kScanChunk = 2048;  // rows per scan chunk (256 threads x 8)
constexpr int kCubeBlocksPerSM = 2;
constexpr int kCubeThreads = 256;

// Per-case data of a binary mask for one spacing (built by k_binary_table).
struct BinCase {
  int ntri;
  unsigned char tri[MC_MAX_TRI][3];  // local edge triples
  int nsum[3];                        // sum of (B - A) x (C - A), local doubled positions
  int tsum;                           // sum of A . (B x C)
  unsigned long long tri4;            // the same triples, 4 bits per edge (nibble 3 t + k)
  double area2;                       // sum of twice the physical triangle areas
};

// ROI of a global row / word: last ROI whose start is <= g.
__device__ __forceinline__ int roi_of_row(const Roi* rois, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rois[mid].row0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int roi_of_word(const Roi* rois, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rois[mid].word0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ const uint32_t* brow(const uint32_t* bits, const Roi& r, int y, int z) {
  return bits + r.word0 + ((long long)(z + 1) * r.BY + (y + 1)) * r.W;
}

__device__ __forceinline__ uint32_t ldw(const uint32_t* row, int w, int W) { return w < W ? row[w] : 0u; }

// ---- pack ------------------------------------------------------------------------

__device__ __forceinline__ uint32_t nz4(uint32_t v) {
  // bit 7 of each byte set iff the byte is non-zero, gathered to 4 bits
  uint32_t t = (v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
  t = (t | v) & 0x80808080u;
  return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// One thread per bitset word of the whole batch (padding rows included).
template <bool SOFT>
__global__ void k_pack(const Roi* rois, int n, long long total, uint32_t* bits,
                       ZeroSet zs) {
  pdl_enter();
  zero_ranges(zs);  // the pass's counters, per-ROI results and scan state
  // every block takes one contiguous range of words, so a thread's words
  // only move forward and its ROI is found by one search and then stepped
  const long long per = ((total + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const long long beg = (long long)blockIdx.x * per, end = min(total, beg + per);
  int ri = 0;
  long long next0 = LLONG_MAX;  // first word of ROI ri + 1
  if (n > 1 && beg + threadIdx.x < end) {
    ri = roi_of_word(rois, n, beg + threadIdx.x);
    next0 = ri + 1 < n ? rois[ri + 1].word0 : LLONG_MAX;
  }
  for (long long id = beg + threadIdx.x; id < end; id += blockDim.x) {
    while (id >= next0) {  // at most a few ROIs per step (ROIs hold whole padded grids)
      ++ri;
      next0 = ri + 1 < n ? rois[ri + 1].word0 : LLONG_MAX;
    }
    const Roi& r = rois[ri];
    // one ROI's words number BY * BZ * W < 2^31 (checked on the host), so the
    // index arithmetic is 32-bit
    const unsigned int local = (unsigned int)(id - r.word0);
    const unsigned int br = local / (unsigned int)r.W;
    const int w = (int)(local - br * (unsigned int)r.W);
    const unsigned int zz = br / (unsigned int)r.BY;
    const int y = (int)(br - zz * (unsigned int)r.BY) - 1, z = (int)zz - 1;
    uint32_t word = 0;
    if (y >= 0 && y < r.ny && z >= 0 && z < r.nz) {
      const int x0 = w * 32;
      const int cnt = min(32, r.nx - x0);
      if (!SOFT) {
        const uint8_t* row = (const uint8_t*)r.data + ((long long)z * r.ny + y) * r.nx;
        if (r.vec16 && cnt == 32) {
          const uint4 a = __ldg(reinterpret_cast<const uint4*>(row + x0));
          const uint4 b = __ldg(reinterpret_cast<const uint4*>(row + x0 + 16));
          word = nz4(a.x) | (nz4(a.y) << 4) | (nz4(a.z) << 8) | (nz4(a.w) << 12) | (nz4(b.x) << 16) |
                 (nz4(b.y) << 20) | (nz4(b.z) << 24) | (nz4(b.w) << 28);
        } else if (r.vec16 && cnt == 16) {
          const uint4 a = __ldg(reinterpret_cast<const uint4*>(row + x0));
          word = nz4(a.x) | (nz4(a.y) << 4) | (nz4(a.z) << 8) | (nz4(a.w) << 12);
        } else {
          // any alignment: the one to three 16-byte blocks holding bytes
          // x0 .. x0 + cnt - 1, realigned by funnel shifts (bytes of the
          // neighbouring rows in them are shifted or masked out); blocks that
          // would reach outside the mask buffer take the byte loop
          const uintptr_t a = reinterpret_cast<uintptr_t>(row + x0);
          const int off = (int)(a & 15u);
          const uint4* blk = reinterpret_cast<const uint4*>(a - (uintptr_t)off);
          const int nblk = (off + cnt + 15) >> 4;
          const uint8_t* base = (const uint8_t*)r.data;
          const uint8_t* end = base + (long long)r.nx * r.ny * r.nz;
          if ((const uint8_t*)blk >= base && (const uint8_t*)(blk + nblk) <= end) {
            const uint4 c0 = __ldg(blk);
            const uint4 c1 = nblk > 1 ? __ldg(blk + 1) : make_uint4(0u, 0u, 0u, 0u);
            const uint4 c2 = nblk > 2 ? __ldg(blk + 2) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t wv[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
            const int j0 = off >> 2, sh = (off & 3) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const uint32_t lo = j0 == 0 ? wv[k] : (j0 == 1 ? wv[k + 1] : (j0 == 2 ? wv[k + 2] : wv[k + 3]));
              const uint32_t hi = j0 == 0 ? wv[k + 1] : (j0 == 1 ? wv[k + 2] : (j0 == 2 ? wv[k + 3] : wv[k + 4]));
              word |= nz4(__funnelshift_r(lo, hi, sh)) << (4 * k);
            }
            if (cnt < 32) word &= (1u << cnt) - 1u;
          } else {
            for (int i = 0; i < cnt; ++i) word |= (uint32_t)(row[x0 + i] != 0) << i;
          }
        }
      } else {
        const float* row = (const float*)r.data + ((long long)z * r.ny + y) * r.nx;
        if (r.vec16 && (cnt & 3) == 0) {
          for (int i = 0; i < cnt; i += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(row + x0 + i));
            word |= ((uint32_t)(v.x > 0.5f) << i) | ((uint32_t)(v.y > 0.5f) << (i + 1)) |
                    ((uint32_t)(v.z > 0.5f) << (i + 2)) | ((uint32_t)(v.w > 0.5f) << (i + 3));
          }
        } else {
          for (int i = 0; i < cnt; ++i) word |= (uint32_t)(row[x0 + i] > 0.5f) << i;
        }
      }
    }
    bits[id] = word;
  }
}

// ---- per-row counts ------------------------------------------------------------------

__device__ __forceinline__ int cube_case(uint32_t r00, uint32_t r00n, uint32_t r10, uint32_t r10n, uint32_t r01,
                                         uint32_t r01n, uint32_t r11, uint32_t r11n, int b) {
  // corner c = cx + 2 cy + 4 cz; rows (cy, cz); "n" words are shifted by one (x + 1)
  return (int)(((r00 >> b) & 1) | (((r00n >> b) & 1) << 1) | (((r10 >> b) & 1) << 2) | (((r10n >> b) & 1) << 3) |
               (((r01 >> b) & 1) << 4) | (((r01n >> b) & 1) << 5) | (((r11 >> b) & 1) << 6) |
               (((r11n >> b) & 1) << 7));
}

__device__ __forceinline__ uint32_t shift1(uint32_t w, uint32_t wn) { return (w >> 1) | (wn << 31); }

// Per-word view of one cube row (y, z): the four mask rows of its cubes and
// the crossing bits of owner row (y, z).
struct WordView {
  uint32_t a, as, b, bs, c, cs, e, es;  // rows (y,z) (y+1,z) (y,z+1) (y+1,z+1), plain and shifted
  uint32_t ex, ey, ez;                  // crossing edges owned by row (y, z)
  uint32_t act;                         // cubes whose corners differ
};

__device__ __forceinline__ WordView word_view(const uint32_t* R00, const uint32_t* R10, const uint32_t* R01,
                                              const uint32_t* R11, int w, int W) {
  WordView v;
  const uint32_t an = ldw(R00, w + 1, W), bn = ldw(R10, w + 1, W), cn = ldw(R01, w + 1, W), en = ldw(R11, w + 1, W);
  v.a = ldw(R00, w, W);
  v.b = ldw(R10, w, W);
  v.c = ldw(R01, w, W);
  v.e = ldw(R11, w, W);
  v.as = shift1(v.a, an);
  v.bs = shift1(v.b, bn);
  v.cs = shift1(v.c, cn);
  v.es = shift1(v.e, en);
  v.ex = v.a ^ v.as;
  v.ey = v.a ^ v.b;
  v.ez = v.a ^ v.c;
  v.act = (v.a | v.b | v.c | v.e | v.as | v.bs | v.cs | v.es) & ~(v.a & v.b & v.c & v.e & v.as & v.bs & v.cs & v.es);
  return v;
}

// Group (L lanes) inclusive scan.
__device__ __forceinline__ int group_incl(int v, int sub, int L) {
  for (int off = 1; off < L; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, v, off, L);
    if (sub >= off) v += o;
  }
  return v;
}

// Row item of a group: global row g, its ROI and (y, z) inside it.
struct RowItem {
  long long g;
  int roi, y, z;
  bool valid;
};

__device__ __forceinline__ RowItem row_item(const Roi* rois, int n, long long total_rows, long long g) {
  RowItem it;
  it.g = g;
  it.valid = g < total_rows;
  it.roi = it.valid ? (n == 1 ? 0 : roi_of_row(rois, n, g)) : 0;
  const Roi& r = rois[it.roi];
  const int local = it.valid ? (int)(g - r.row0) : 0;  // rows of one ROI < 2^31
  it.y = it.valid ? local % (r.ny + 1) - 1 : -1;
  it.z = it.valid ? local / (r.ny + 1) - 1 : -1;
  return it;
}

// One group of L lanes per row item (y, z) in [-1, ny-1] x [-1, nz-1] of each ROI:
//   counts = (vertices owned by the row, triangles of the cube row, inside voxels, active cubes)
//   wpre[row][w] = vertices of the row owned by x < 32 w (row-local prefix)
//   tpre[row][w] = triangles of the cube row's cubes x < 32 w (row-local prefix)
// and every word with crossings or active cubes (word 0 also for the x = -1
// vertex and cube) is appended to wlist (any order: the prefixes fix the ids).
constexpr int kCountThreads = 256;
__global__ void __launch_bounds__(kCountThreads) k_count(const uint32_t* bits, const Roi* rois, int n, long long total_rows,
                        int L, int Wc, int4* counts, int* wpre, int* tpre,
                        int2* wlist, long long wlist_cap, MeshTotals* tot) {
  pdl_enter();
  const int lane = threadIdx.x & 31, sub = lane % L, gpw = 32 / L;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  // list entries are staged per warp and reserved 33..64 at a time
  __shared__ int2 s_lb[kCountThreads / 32][64];
  int2* lb = s_lb[threadIdx.x >> 5];
  int lbn = 0;
  auto list_flush = [&]() {
    __syncwarp();
    long long lbase = 0;
    if (lane == 0) lbase = (long long)atomicAdd((unsigned long long*)&tot->nwords, (unsigned long long)lbn);
    lbase = __shfl_sync(0xffffffffu, lbase, 0);
    for (int i = lane; i < lbn; i += 32)
      if (lbase + i < wlist_cap) wlist[lbase + i] = lb[i];
    __syncwarp();
    lbn = 0;
  };
  for (long long base = warp * gpw; base < total_rows; base += nwarps * gpw) {
    const RowItem it = row_item(rois, n, total_rows, base + lane / L);
    const Roi& r = rois[it.roi];
    const int y = it.y, z = it.z, W = r.W;
    const uint32_t* R00 = brow(bits, r, y, z);
    const uint32_t* R10 = brow(bits, r, y + 1, z);
    const uint32_t* R01 = brow(bits, r, y, z + 1);
    const uint32_t* R11 = brow(bits, r, y + 1, z + 1);
    // owner x = -1 and cube x = -1 (corners cx = 1 at voxel x = 0)
    const uint32_t a0 = ldw(R00, 0, W) & 1u, b0 = ldw(R10, 0, W) & 1u, c0 = ldw(R01, 0, W) & 1u,
                   e0 = ldw(R11, 0, W) & 1u;
    const int case_m1 = (int)((a0 << 1) | (b0 << 3) | (c0 << 5) | (e0 << 7));
    int carry = (int)a0;
    int tcarry = MC_CASE_NTRI[case_m1];
    int nt = sub == 0 ? tcarry : 0;
    int na = (sub == 0 && case_m1) ? 1 : 0;
    int nvox = 0;
    const long long wbase = r.wpre0 + (it.g - r.row0) * (long long)W;
    for (int w = sub; w < Wc; w += L) {  // the same trip count on every lane (Wc is a multiple of L)
      const WordView v = word_view(R00, R10, R01, R11, w, W);
      // no crossing, no active cube and no x = -1 entry in any of the warp's
      // words: nothing to count, scan or list, only the inside voxels
      const bool quiet = (v.ex | v.ey | v.ez | v.act) == 0u && !(w == 0 && (a0 || case_m1));
      if (__all_sync(0xffffffffu, quiet)) {
        if (y >= 0 && z >= 0) nvox += __popc(v.a);
        continue;
      }
      const int cnt = __popc(v.ex) + __popc(v.ey) + __popc(v.ez);
      int tw = 0;
      for (uint32_t act = v.act; act; act &= act - 1)
        tw += MC_CASE_NTRI[cube_case(v.a, v.as, v.b, v.bs, v.c, v.cs, v.e, v.es, __ffs(act) - 1)];
      const int incl = group_incl(cnt, sub, L), tincl = group_incl(tw, sub, L);
      const bool live = it.valid && w < W;
      // words with surface go to the emit list; only their prefixes are ever
      // read (a cube's edge is owned by a word with a crossing, i.e. listed)
      const bool surf = live && ((v.ex | v.ey | v.ez | v.act) != 0u || (w == 0 && (a0 || case_m1)));
      if (surf) {
        wpre[wbase + w] = carry + incl - cnt;
        tpre[wbase + w] = tcarry + tincl - tw;
      }
      carry += __shfl_sync(0xffffffffu, incl, L - 1, L);
      tcarry += __shfl_sync(0xffffffffu, tincl, L - 1, L);
      if (y >= 0 && z >= 0) nvox += __popc(v.a);
      na += __popc(v.act);
      nt += tw;
      const unsigned int sm = __ballot_sync(0xffffffffu, surf);
      if (sm) {
        if (surf) lb[lbn + __popc(sm & ((1u << lane) - 1u))] = make_int2((int)(it.g), w);
        lbn += __popc(sm);
        if (lbn > 32) list_flush();
      }
    }
    for (int off = L / 2; off > 0; off >>= 1) {
      nt += __shfl_xor_sync(0xffffffffu, nt, off, L);
      nvox += __shfl_xor_sync(0xffffffffu, nvox, off, L);
      na += __shfl_xor_sync(0xffffffffu, na, off, L);
    }
    if (it.valid && sub == 0) counts[it.g] = make_int4(carry, nt, nvox, na);
  }
  if (lbn) list_flush();
}

// ---- scan of row counts -------------------------------------------------------------
// One kernel, decoupled look-back over chunks of kScanChunk rows: prefix[4 r + q]
// = global exclusive prefix of (vertices, triangles, active cubes, inside
// voxels) at row r over the whole batch; the last chunk writes the totals and
// the last block to finish derives every ROI's id ranges.

__global__ void k_scan_rows(const int4* counts, long long R, int nchunks, long long* prefix,
                            ScanTile<4>* tiles, unsigned int* tick,
                            MeshTotals* tot, const Roi* rois, int n,
                            RoiOut* out) {
  pdl_enter();
  __shared__ long long sw[4][8];
  __shared__ long long s_ex[4];
  __shared__ int s_c;
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_c = (int)atomicAdd(&tick[0], 1u);
  __syncthreads();
  const int c = s_c;
  const long long beg = (long long)c * kScanChunk;
  constexpr int per = kScanChunk / 256;
  long long own[4] = {0, 0, 0, 0};
  int4 cv[per];
  for (int i = 0; i < per; ++i) {
    const long long r = beg + threadIdx.x * per + i;
    cv[i] = r < R ? counts[r] : make_int4(0, 0, 0, 0);
    own[0] += cv[i].x; own[1] += cv[i].y; own[2] += cv[i].w; own[3] += cv[i].z;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc[4] = {own[0], own[1], own[2], own[3]};
  for (int off = 1; off < 32; off <<= 1)
    for (int q = 0; q < 4; ++q) {
      const long long o = __shfl_up_sync(0xffffffffu, inc[q], off);
      if (lane >= off) inc[q] += o;
    }
  if (lane == 31)
    for (int q = 0; q < 4; ++q) sw[q][wid] = inc[q];
  __syncthreads();
  long long ex[4], agg[4];
  for (int q = 0; q < 4; ++q) {
    long long wb = 0, tb = 0;
    for (int k = 0; k < 8; ++k) {
      if (k < wid) wb += sw[q][k];
      tb += sw[q][k];
    }
    ex[q] = wb + inc[q] - own[q];
    agg[q] = tb;
  }
  if (threadIdx.x == 0) scan_publish(&tiles[c], agg, c == 0 ? 2ull : 1ull);
  if (wid == 0) {
    long long e[4] = {0, 0, 0, 0};
    if (c > 0) {
      scan_lookback(tiles, c, e, &tot->status);
      if (lane == 0) {
        long long incl[4];
        for (int q = 0; q < 4; ++q) incl[q] = e[q] + agg[q];
        scan_publish(&tiles[c], incl, 2ull);
      }
    }
    if (lane == 0)
      for (int q = 0; q < 4; ++q) s_ex[q] = e[q];
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q) ex[q] += s_ex[q];
  for (int i = 0; i < per; ++i) {
    const long long r = beg + threadIdx.x * per + i;
    if (r < R)
      for (int q = 0; q < 4; ++q) prefix[4 * r + q] = ex[q];
    ex[0] += cv[i].x; ex[1] += cv[i].y; ex[2] += cv[i].w; ex[3] += cv[i].z;
  }
  if (c == nchunks - 1 && threadIdx.x == 0) {
    tot->nv = s_ex[0] + agg[0];
    tot->nt = s_ex[1] + agg[1];
    tot->na = s_ex[2] + agg[2];
    tot->nvox = s_ex[3] + agg[3];
  }
  // the last block to finish: id ranges of every ROI
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tick[1], 1u) == (unsigned int)nchunks - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const Roi& r = rois[i];
    const bool last = i == n - 1;
    const long long e = r.row0 + r.R;
    RoiOut o = out[i];
    o.v0 = __ldcg(&prefix[4 * r.row0]);
    o.t0 = __ldcg(&prefix[4 * r.row0 + 1]);
    o.c0 = __ldcg(&prefix[4 * r.row0 + 2]);
    const long long x0 = __ldcg(&prefix[4 * r.row0 + 3]);
    o.nv = (last ? __ldcg(&tot->nv) : __ldcg(&prefix[4 * e])) - o.v0;
    o.nt = (last ? __ldcg(&tot->nt) : __ldcg(&prefix[4 * e + 1])) - o.t0;
    o.na = (last ? __ldcg(&tot->na) : __ldcg(&prefix[4 * e + 2])) - o.c0;
    o.nvox = (last ? __ldcg(&tot->nvox) : __ldcg(&prefix[4 * e + 3])) - x0;
    out[i] = o;
  }
}

// q: 0 vertices, 1 triangles, 2 active cubes, 3 inside voxels (global exclusive prefixes)
__device__ __forceinline__ long long row_base(const long long* prefix, long long r, int q) {
  return prefix[4 * r + q];
}

// ---- triangulation choice -----------------------------------------------------------
// Among a loop's admissible candidates (stored in ascending lexicographic order
// of their canonical triple lists): minimum area score, then maximum volume,
// then the first in list order.  Pinned FP64 arithmetic, so the same choice
// as any other implementation of the rule.  Volumes are computed only when
// the scores leave a tie (they decide nothing otherwise).
__device__ int select_candidate(int loop, const double (*w)[3], const double* sp) {
  const int k = MC_LOOP_K[loop], nt = k - 2;
  const int cb = MC_LOOP_CAND_BEGIN[loop], ce = MC_LOOP_CAND_BEGIN[loop + 1];
  if (ce - cb == 1) return cb;
  double sc[MC_MAX_CAND];
  double smin = 0.0;
  for (int c = cb; c < ce; ++c) {
    const int tb = MC_CAND_TRI_BEGIN[c];
    double s = 0.0;
    for (int t = 0; t < nt; ++t) {
      const unsigned char* tr = &MC_CAND_TRIPLES[3 * (tb + t)];
      s = __dadd_rn(s, pin_tri_r(w[tr[0]], w[tr[1]], w[tr[2]]));
    }
    sc[c - cb] = s;
    if (c == cb || s < smin) smin = s;
  }
  const double slim = __dadd_rn(smin, __dmul_rn(smin, 1e-12));
  int tied = 0, only = cb;
  for (int c = 0; c < ce - cb; ++c)
    if (sc[c] <= slim) { ++tied; only = cb + c; }
  if (tied == 1) return only;
  double vv[MC_MAX_CAND];
  double vmax = 0.0;
  bool have = false;
  for (int c = 0; c < ce - cb; ++c) {
    if (!(sc[c] <= slim)) continue;
    const int tb = MC_CAND_TRI_BEGIN[cb + c];
    double v = 0.0;
    for (int t = 0; t < nt; ++t) {
      const unsigned char* tr = &MC_CAND_TRIPLES[3 * (tb + t)];
      v = __dadd_rn(v, pin_vol6(w[tr[0]], w[tr[1]], w[tr[2]]));
    }
    vv[c] = v;
    if (!have || v > vmax) { vmax = v; have = true; }
  }
  const double vlim = __dsub_rn(vmax, __dmul_rn(__dmul_rn(__dmul_rn(sp[0], sp[1]), sp[2]), 1e-9));
  for (int c = 0; c < ce - cb; ++c)
    if (sc[c] <= slim && vv[c] >= vlim) return cb + c;
  return cb;  // not reached
}

// Binary masks: every crossing sits at an edge midpoint, so the choice depends
// only on (case, spacing).  One thread per case writes its triangles (local
// edge triples) and the per-case sums used for volume and area:
//   nsum = sum over the case's triangles of (B - A) x (C - A),
//   tsum = sum of A . (B x C),
// with A, B, C the local doubled positions (integers 0..2), and area2 = sum of
// |cof(H) ((B - A) x (C - A))| with H = diag(s / 2).
__global__ void k_binary_table(const double* spacings, BinCase* tabs) {
  pdl_enter();
  const int cs = threadIdx.x;
  const double sx = spacings[3 * blockIdx.x], sy = spacings[3 * blockIdx.x + 1], sz = spacings[3 * blockIdx.x + 2];
  BinCase* tab = tabs + 256 * blockIdx.x;
  const double sp[3] = {sx, sy, sz};
  double w[12][3];
  int lp[12][3];
  for (int e = 0; e < 12; ++e) {
    const int c = MC_EDGE_CORNER[e], a = MC_EDGE_AXIS[e];
    for (int k = 0; k < 3; ++k) {
      w[e][k] = __dmul_rn(__dadd_rn((double)((c >> k) & 1), k == a ? 0.5 : 0.0), sp[k]);
      lp[e][k] = 2 * ((c >> k) & 1) + (k == a);
    }
  }
  BinCase out;
  out.ntri = 0;
  out.tri4 = 0ull;
  out.nsum[0] = out.nsum[1] = out.nsum[2] = 0;
  out.tsum = 0;
  out.area2 = 0.0;
  const double hx = 0.5 * sx, hy = 0.5 * sy, hz = 0.5 * sz;
  const double cof[3] = {hy * hz, hx * hz, hx * hy};
  for (int l = MC_CASE_LOOP_BEGIN[cs]; l < MC_CASE_LOOP_BEGIN[cs + 1]; ++l) {
    const int c = select_candidate(l, w, sp);
    const int tb = MC_CAND_TRI_BEGIN[c];
    for (int t = 0; t < MC_LOOP_K[l] - 2; ++t) {
      const int e0 = MC_CAND_TRIPLES[3 * (tb + t)], e1 = MC_CAND_TRIPLES[3 * (tb + t) + 1],
                e2 = MC_CAND_TRIPLES[3 * (tb + t) + 2];
      out.tri[out.ntri][0] = (unsigned char)e0;
      out.tri[out.ntri][1] = (unsigned char)e1;
      out.tri[out.ntri][2] = (unsigned char)e2;
      out.tri4 |= ((unsigned long long)e0 | ((unsigned long long)e1 << 4) | ((unsigned long long)e2 << 8))
                  << (12 * out.ntri);
      out.ntri++;
      const int* A = lp[e0];
      const int* B = lp[e1];
      const int* C = lp[e2];
      const int u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      const int n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
      for (int k = 0; k < 3; ++k) out.nsum[k] += n[k];
      out.tsum += A[0] * (B[1] * C[2] - B[2] * C[1]) + A[1] * (B[2] * C[0] - B[0] * C[2]) +
                  A[2] * (B[0] * C[1] - B[1] * C[0]);
      const double fx = cof[0] * n[0], fy = cof[1] * n[1], fz = cof[2] * n[2];
      out.area2 += sqrt(fx * fx + fy * fy + fz * fz);
    }
  }
  tab[cs] = out;
}

__device__ __forceinline__ float value_at(const Roi& r, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= r.nx || y >= r.ny || z >= r.nz) return 0.0f;
  return __ldg((const float*)r.data + ((long long)z * r.ny + y) * r.nx + x);
}

__device__ __forceinline__ double crossing_t(double v0, double v1) {
  return __ddiv_rn(__dsub_rn(0.5, v0), __dsub_rn(v1, v0));
}

// ---- rows: vertices and the active-cube list --------------------------------------------

template <bool SOFT>
__global__ void k_rows(const uint32_t* bits, const Roi* rois, int n, long long total_rows,
                       int L, int Wc, const int4* counts, const int* wpre,
                       const long long* prefix, int16_t* idx2, double* vt, int4* cubes, long long vcap,
                       long long ccap, MeshTotals* tot) {
  pdl_enter();
  const int lane = threadIdx.x & 31, sub = lane % L, gpw = 32 / L;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned int err = 0;
  for (long long base = warp * gpw; base < total_rows; base += nwarps * gpw) {
    const RowItem it = row_item(rois, n, total_rows, base + lane / L);
    // rows without vertices and active cubes have nothing to write; skip
    // them when the whole warp agrees (the group scans below are warp-wide)
    const int4 rc = it.valid ? counts[it.g] : make_int4(0, 0, 0, 0);
    if (__all_sync(0xffffffffu, rc.x == 0 && rc.w == 0)) continue;
    const Roi& r = rois[it.roi];
    const int y = it.y, z = it.z, W = r.W;
    const uint32_t* R00 = brow(bits, r, y, z);
    const uint32_t* R10 = brow(bits, r, y + 1, z);
    const uint32_t* R01 = brow(bits, r, y, z + 1);
    const uint32_t* R11 = brow(bits, r, y + 1, z + 1);
    const long long vb = it.valid ? row_base(prefix, it.g, 0) : 0;
    const long long tb = it.valid ? row_base(prefix, it.g, 1) : 0;
    const long long cb = it.valid ? row_base(prefix, it.g, 2) : 0;
    const uint32_t a0 = ldw(R00, 0, W) & 1u, b0 = ldw(R10, 0, W) & 1u, c0 = ldw(R01, 0, W) & 1u,
                   e0 = ldw(R11, 0, W) & 1u;
    const int case_m1 = (int)((a0 << 1) | (b0 << 3) | (c0 << 5) | (e0 << 7));
    const int nt_m1 = MC_CASE_NTRI[case_m1], na_m1 = case_m1 ? 1 : 0;
    if (it.valid && sub == 0) {
      if (a0) {  // owner x = -1: x-edge into voxel 0, the row's first vertex
        if (vb < vcap) {
          idx2[3 * vb] = (int16_t)(-1);
          idx2[3 * vb + 1] = (int16_t)(2 * y);
          idx2[3 * vb + 2] = (int16_t)(2 * z);
          if (SOFT) vt[vb] = crossing_t(0.0, (double)value_at(r, 0, y, z));
        } else {
          err |= DEV_ERR_VCAP;
        }
      }
      if (na_m1) {
        if (cb < ccap) cubes[cb] = make_int4(-1, (int)it.g, case_m1, (int)tb);
        else err |= DEV_ERR_TCAP;
      }
    }
    int carry_t = nt_m1, carry_c = na_m1;
    const long long wbase = r.wpre0 + (it.g - r.row0) * (long long)W;
    for (int w = sub; w < Wc; w += L) {
      const WordView v = word_view(R00, R10, R01, R11, w, W);
      int tcnt = 0;
      for (uint32_t act = v.act; act; act &= act - 1)
        tcnt += MC_CASE_NTRI[cube_case(v.a, v.as, v.b, v.bs, v.c, v.cs, v.e, v.es, __ffs(act) - 1)];
      const int ccnt = __popc(v.act);
      const int ti = group_incl(tcnt, sub, L), ci = group_incl(ccnt, sub, L);
      long long tid = tb + carry_t + ti - tcnt;
      long long cid = cb + carry_c + ci - ccnt;
      carry_t += __shfl_sync(0xffffffffu, ti, L - 1, L);
      carry_c += __shfl_sync(0xffffffffu, ci, L - 1, L);
      if (!it.valid || w >= W) continue;
      // vertices owned by (x, y, z), x in this word, canonical (x, axis) order
      long long id = vb + wpre[wbase + w];
      for (uint32_t u = v.ex | v.ey | v.ez; u; u &= u - 1) {
        const int bit = __ffs(u) - 1, x = 32 * w + bit;
        for (int a = 0; a < 3; ++a) {
          const uint32_t eb = a == 0 ? v.ex : (a == 1 ? v.ey : v.ez);
          if (!((eb >> bit) & 1u)) continue;
          if (id < vcap) {
            idx2[3 * id] = (int16_t)(2 * x + (a == 0));
            idx2[3 * id + 1] = (int16_t)(2 * y + (a == 1));
            idx2[3 * id + 2] = (int16_t)(2 * z + (a == 2));
            if (SOFT) {
              const double v0 = (double)value_at(r, x, y, z);
              const double v1 = (double)value_at(r, x + (a == 0), y + (a == 1), z + (a == 2));
              vt[id] = crossing_t(v0, v1);
            }
          } else {
            err |= DEV_ERR_VCAP;
          }
          ++id;
        }
      }
      // active cubes of this word, ascending x
      for (uint32_t act = v.act; act; act &= act - 1) {
        const int bit = __ffs(act) - 1;
        const int cs = cube_case(v.a, v.as, v.b, v.bs, v.c, v.cs, v.e, v.es, bit);
        if (cid < ccap) cubes[cid] = make_int4(32 * w + bit, (int)it.g, cs, (int)tid);
        else err |= DEV_ERR_TCAP;
        ++cid;
        tid += MC_CASE_NTRI[cs];
      }
    }
  }
  if (err) atomicOr(&tot->status, err);
}

// ---- cubes: triangles, volume, area -------------------------------------------------------

// Crossing-edge info of one owner row at one word: crossing bits and the
// row-local vertex prefix of the word, plus the row's first vertex id.
struct OwnerWord {
  long long base;
  int pre;
  uint32_t ex, ey, ez;
};

__device__ __forceinline__ OwnerWord owner_word(const uint32_t* bits, const Roi& r, const int* wpre,
                                                const long long* prefix, int xo, int yo, int zo) {
  OwnerWord o;
  const long long g = r.row0 + (long long)(zo + 1) * (r.ny + 1) + (yo + 1);
  o.base = row_base(prefix, g, 0);
  if (xo < 0) {
    o.pre = 0; o.ex = o.ey = o.ez = 0u;
    return o;
  }
  const int w = xo >> 5;
  const uint32_t* R0 = brow(bits, r, yo, zo);
  const uint32_t b = R0[w], bn = ldw(R0, w + 1, r.W);
  o.ex = b ^ shift1(b, bn);
  o.ey = b ^ brow(bits, r, yo + 1, zo)[w];
  o.ez = b ^ brow(bits, r, yo, zo + 1)[w];
  o.pre = wpre[r.wpre0 + (g - r.row0) * (long long)r.W + w];
  return o;
}

__device__ __forceinline__ int owner_rank(const OwnerWord& o, int xo, int a) {
  if (xo < 0) return 0;  // the x-edge into voxel 0 is the row's first vertex
  const int bit = xo & 31;
  const uint32_t low = (1u << bit) - 1u;
  int rk = o.pre + __popc(o.ex & low) + __popc(o.ey & low) + __popc(o.ez & low);
  if (a >= 1) rk += (o.ex >> bit) & 1u;
  if (a >= 2) rk += (o.ey >> bit) & 1u;
  return rk;
}

// Local edge e = (corner, axis) in canonical (cz, cy, cx, axis) order.
__device__ __forceinline__ int edge_corner(int e) {
  return e < 3 ? 0 : (e < 5 ? 1 : (e < 7 ? 2 : (e < 8 ? 3 : (e < 10 ? 4 : (e < 11 ? 5 : 6)))));
}
__device__ __forceinline__ int edge_axis(int e) {
  constexpr unsigned long long kAxes = (0ull << 0) | (1ull << 2) | (2ull << 4) | (1ull << 6) | (2ull << 8) |
                                      (0ull << 10) | (2ull << 12) | (2ull << 14) | (0ull << 16) | (1ull << 18) |
                                      (1ull << 20) | (0ull << 22);
  return (int)((kAxes >> (2 * e)) & 3ull);
}

template <bool SOFT>
__global__ void __launch_bounds__(kCubeThreads) k_cubes(const uint32_t* bits, const Roi* rois,
                                                        int n, const int* wpre,
                                                        const long long* prefix,
                                                        const int4* cubes, const BinCase* tab,
                                                        int32_t* tri, long long ccap, long long tcap,
                                                        MeshTotals* tot, RoiOut* out,
                                                        unsigned long long* case_hist,
                                                        double* partial) {
  pdl_enter();
  const long long ncubes = min(tot->na, ccap);
  long long vsum = 0;
  double acc_v6 = 0.0, acc_a2 = 0.0;
  unsigned int err = 0;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // warp-uniform loop: lanes past the end take part in the aggregation below.
  // Consecutive 32-cube groups go to consecutive blocks (the warps are
  // interleaved over the grid), so a short cube list still spreads over every
  // SM's FP64 units instead of filling the first blocks only.
  const long long gw = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (long long k0 = gw * 32; k0 < ncubes; k0 += stride) {
    const long long k = k0 + lane;
    const bool valid = k < ncubes;
    const int4 cu = valid ? cubes[k] : make_int4(0, 0, 0, 0);
    const int roi = valid ? (n == 1 ? 0 : roi_of_row(rois, n, cu.y)) : 0;
    int cs = cu.z;
    if (valid) {
      const Roi& r = rois[roi];
      const int x = cu.x;
      const int local = (int)(cu.y - r.row0);
      const int y = local % (r.ny + 1) - 1, z = local / (r.ny + 1) - 1;
      const double sp[3] = {r.sx, r.sy, r.sz};
      const int nn[3] = {r.nx, r.ny, r.nz};
      const unsigned int emask = MC_CASE_EDGES[cs];
      // owner rows (cy, cz) at the word of x (cx = 0) or of x + 1 (cx = 1), each loaded once
      OwnerWord ow[8];
      unsigned int have = 0;
      int vid[12];
      double P[12][3], wl[12][3];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        if (!((emask >> e) & 1u)) continue;
        const int c = edge_corner(e), a = edge_axis(e);
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const int slot = cz * 4 + cy * 2 + cx;
        const int g[3] = {x + cx, y + cy, z + cz};
        if (!((have >> slot) & 1u)) {
          ow[slot] = owner_word(bits, r, wpre, prefix, g[0], g[1], g[2]);
          have |= 1u << slot;
        }
        vid[e] = (int)(ow[slot].base + owner_rank(ow[slot], g[0], a));
        if (SOFT) {
          const double v0 = (double)value_at(r, g[0], g[1], g[2]);
          const double v1 = (double)value_at(r, g[0] + (a == 0), g[1] + (a == 1), g[2] + (a == 2));
          const double t = crossing_t(v0, v1);
          for (int q = 0; q < 3; ++q) {
            P[e][q] = ((double)g[q] - 0.5 * (double)(nn[q] - 1) + (q == a ? t : 0.0)) * sp[q];
            wl[e][q] = __dmul_rn(__dadd_rn((double)((c >> q) & 1), q == a ? t : 0.0), sp[q]);
          }
        }
      }
      long long tid = cu.w;
      if (SOFT) {
        for (int l = MC_CASE_LOOP_BEGIN[cs]; l < MC_CASE_LOOP_BEGIN[cs + 1]; ++l) {
          const int cand = select_candidate(l, wl, sp);
          const int tb2 = MC_CAND_TRI_BEGIN[cand];
          for (int t = 0; t < MC_LOOP_K[l] - 2; ++t, ++tid) {
            const int e0 = MC_CAND_TRIPLES[3 * (tb2 + t)], e1 = MC_CAND_TRIPLES[3 * (tb2 + t) + 1],
                      e2 = MC_CAND_TRIPLES[3 * (tb2 + t) + 2];
            if (tid < tcap) {
              tri[3 * tid] = vid[e0];
              tri[3 * tid + 1] = vid[e1];
              tri[3 * tid + 2] = vid[e2];
            } else {
              err |= DEV_ERR_TCAP;
            }
            const double* A = P[e0];
            const double* B = P[e1];
            const double* C = P[e2];
            acc_v6 += A[0] * (B[1] * C[2] - B[2] * C[1]) + A[1] * (B[2] * C[0] - B[0] * C[2]) +
                      A[2] * (B[0] * C[1] - B[1] * C[0]);
            const double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
            const double vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
            const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
            acc_a2 += sqrt(nx * nx + ny * ny + nz * nz);
          }
        }
      } else {
        const BinCase& bc = tab[r.tab * 256 + cs];
        for (int t = 0; t < bc.ntri; ++t, ++tid) {
          if (tid < tcap) {
            tri[3 * tid] = vid[bc.tri[t][0]];
            tri[3 * tid + 1] = vid[bc.tri[t][1]];
            tri[3 * tid + 2] = vid[bc.tri[t][2]];
          } else {
            err |= DEV_ERR_TCAP;
          }
        }
        // exact volume: positions in half-voxel units relative to the padded-box
        // centre, P = o + local; sum A.(B x C) = o . nsum + tsum
        const long long ox = 2LL * x - (r.nx - 1), oy = 2LL * y - (r.ny - 1), oz = 2LL * z - (r.nz - 1);
        vsum = ox * bc.nsum[0] + oy * bc.nsum[1] + oz * bc.nsum[2] + bc.tsum;
      }
    }
    if (SOFT && n > 1) {
      // a batch of soft maps: per-ROI sums by FP64 atomics (one per warp
      // when its lanes share the ROI), the closed forms at the end
      const unsigned int same_roi = __match_any_sync(0xffffffffu, valid ? roi : -1);
      if (same_roi == 0xffffffffu) {
        for (int off = 16; off > 0; off >>= 1) {
          acc_v6 += __shfl_xor_sync(0xffffffffu, acc_v6, off);
          acc_a2 += __shfl_xor_sync(0xffffffffu, acc_a2, off);
        }
        if (lane == 0 && valid) {
          atomicAdd(&out[roi].vol6, acc_v6);
          atomicAdd(&out[roi].area2, acc_a2);
        }
      } else if (valid) {
        atomicAdd(&out[roi].vol6, acc_v6);
        atomicAdd(&out[roi].area2, acc_a2);
      }
      acc_v6 = 0.0;
      acc_a2 = 0.0;
    }
    if (!SOFT) {
      // lanes of one ROI add their volume sums with one atomic; lanes of one
      // (ROI, case) add their count with one atomic
      // |vsum| of one cube < 5e6, so a warp's sum fits in 32 bits
      const unsigned int same_roi = __match_any_sync(0xffffffffu, valid ? roi : -1);
      const int vs = __reduce_add_sync(same_roi, (int)vsum);
      if (valid && lane == __ffs(same_roi) - 1 && vs)
        atomicAdd((unsigned long long*)&out[roi].vsum, (unsigned long long)(long long)vs);
      const long long key = valid ? (long long)roi * 256 + cs : -1;
      const unsigned int same_case = __match_any_sync(0xffffffffu, key);
      if (valid && lane == __ffs(same_case) - 1) atomicAdd(&case_hist[key], (unsigned long long)__popc(same_case));
      vsum = 0;
    }
  }
  if (err) atomicOr(&tot->status, err);
  if (!SOFT) return;
  __shared__ bool last;
  if (n > 1) {  // the last CTA: closed forms of every map of the batch
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&tot->done_ctas, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      closed_form_features(__ldcg(&out[i].vol6) / 6.0, __ldcg(&out[i].area2) * 0.5, out[i].derived);
      out[i].has_derived = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) tot->done_ctas = 0;
    return;
  }
  // soft map (one ROI): fixed-order block reduction, then the last CTA finishes
  const int wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    acc_v6 += __shfl_xor_sync(0xffffffffu, acc_v6, off);
    acc_a2 += __shfl_xor_sync(0xffffffffu, acc_a2, off);
  }
  __shared__ double s_v6[kCubeThreads / 32], s_a2[kCubeThreads / 32];
  if (lane == 0) { s_v6[wid] = acc_v6; s_a2[wid] = acc_a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b6 = 0.0, b2 = 0.0;
    for (int k2 = 0; k2 < kCubeThreads / 32; ++k2) { b6 += s_v6[k2]; b2 += s_a2[k2]; }
    partial[2 * blockIdx.x] = b6;
    partial[2 * blockIdx.x + 1] = b2;
    __threadfence();
    last = atomicAdd(&tot->done_ctas, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double v = 0.0, a = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      v += __ldcg(&partial[2 * b]);
      a += __ldcg(&partial[2 * b + 1]);
    }
    out[0].vol6 = v;
    out[0].area2 = a;
    closed_form_features(v / 6.0, a * 0.5, out[0].derived);
    out[0].has_derived = 1;
    tot->done_ctas = 0;
  }
}

// ---- binary masks: vertices and triangles of the words with surface ----------------
// Warps take chunks of 32 listed words from a ticket (any order: the row bases
// and the row-local word prefixes fix every id), one word per lane.  Each lane
// loads its word's cube rows and the crossing masks and vertex prefixes of the
// four owner rows (y, z), (y+1, z), (y, z+1), (y+1, z+1) into shared memory
// (one array per quantity, so lanes hit distinct banks), plus the bit-0
// crossings and prefixes of the next word for cubes at bit 31.  The warp then
// lists the crossing positions and the active cubes of its 32 words and works
// through each list 32 entries at a time, every lane taking one entry, so a
// word with a long run of surface is shared by the whole warp.  A vertex id is
// its row base + word prefix + rank in the word.  A cube's twelve edge ids
// come branch-free from the owner rows' prefixes at x and x + 1; its triangle
// ids are its word's base + the triangles of the word's earlier cubes (a
// prefix over the cube's run in the list plus a per-word carry between rounds).
constexpr int kEmitThreads = 128;
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kEmitBlocksPerSM = 6;  // 36.3 KB of shared memory per block
constexpr int kListCap = 32 * 33;   // 32 words x (32 bits + the x = -1 entry)

struct __align__(16) EmitShared {
  uint32_t cw[8][32];  // per lane: rows (y,z) (y+1,z) (y,z+1) (y+1,z+1) at x and x + 1: a, as, b, bs, c, cs, e, es
  int4 own[4][32];     // per owner row, per lane: ex, ey, ez, row-local vertex prefix of the word
  int onx[4][32];      // per owner row: next word's prefix << 2 | ey bit 0 << 1 | ex bit 0
  int vb[4][32];       // first vertex id of the owner rows
  long long tb[32];    // first triangle id of the word's cubes
  int y[32], z[32], wd[32], roi[32], tab[32], tcar[32];
  int vid[12][32];     // edge vertex ids of the cube each lane is working on
  unsigned short list[kListCap];
};

__device__ __forceinline__ int warp_incl(int v, int lane) {
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  return v;
}

// Local edge e = (corner, axis) in canonical (cz, cy, cx, axis) order, as packed constants.
constexpr unsigned long long kEdgeCorner = 0ull | (0ull << 3) | (0ull << 6) | (1ull << 9) | (1ull << 12) |
                                           (2ull << 15) | (2ull << 18) | (3ull << 21) | (4ull << 24) |
                                           (4ull << 27) | (5ull << 30) | (6ull << 33);
constexpr unsigned int kEdgeAxis = (0u << 0) | (1u << 2) | (2u << 4) | (1u << 6) | (2u << 8) | (0u << 10) |
                                   (2u << 12) | (2u << 14) | (0u << 16) | (1u << 18) | (1u << 20) | (0u << 22);

__global__ void __launch_bounds__(kEmitThreads, kEmitBlocksPerSM)
    k_emit(const uint32_t* bits, const Roi* rois, int n, const int2* wlist,
           long long wlist_cap, const int* wpre, const int* tpre,
           const long long* prefix, const BinCase* tab,
           int16_t* idx2, int32_t* tri, long long vcap, long long tcap,
           MeshTotals* tot, RoiOut* out, unsigned long long* case_hist) {
  pdl_enter();
  __shared__ EmitShared sh[kEmitWarps];
  // case counts of the warp's current ROI, 16 bits each: they are flushed
  // before the cubes counted since the last flush could pass 65,535
  __shared__ unsigned short s_hist[kEmitWarps][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  EmitShared& S = sh[wid];
  unsigned short* hist = s_hist[wid];
  unsigned int since = 0;  // cubes of the tagged ROI offered to the counts since the last flush
  const long long nlist = min(tot->nwords, wlist_cap);
  const long long nchunk = (nlist + 31) / 32;
  unsigned int err = 0;
  // volume sum and case counts of one ROI (tag) stay in the warp until the ROI changes
  int tag = -1;
  long long vacc = 0;
  for (int c = lane; c < 256; c += 32) hist[c] = 0;
  auto flush = [&]() {
    __syncwarp();
    if (tag >= 0) {
      for (int c = lane; c < 256; c += 32) {
        const unsigned int h = hist[c];
        if (h) atomicAdd(&case_hist[(long long)tag * 256 + c], (unsigned long long)h);
        hist[c] = 0;
      }
      long long v = vacc;  // the leader of the tagged run differs between rounds
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0 && v) atomicAdd((unsigned long long*)&out[tag].vsum, (unsigned long long)v);
    }
    vacc = 0;
    __syncwarp();
  };
  while (true) {
    unsigned long long ch = 0;
    if (lane == 0) ch = atomicAdd(&tot->emit_ticket, 1ull);
    ch = __shfl_sync(0xffffffffu, ch, 0);
    if ((long long)ch >= nchunk) break;  // warp-uniform
    const long long k = (long long)ch * 32 + lane;
    const bool valid = k < nlist;
    uint32_t u = 0, act = 0;
    bool m1v = false;
    int case_m1 = 0;
    {
      const int2 en = valid ? wlist[k] : make_int2(0, 0);
      const long long g = en.x;
      const int w = en.y;
      const int roi = valid ? (n == 1 ? 0 : roi_of_row(rois, n, g)) : 0;
      const Roi& r = rois[roi];
      const int W = r.W;
      const int local = (int)(g - r.row0);
      const int y = local % (r.ny + 1) - 1, z = local / (r.ny + 1) - 1;
      const bool oky = y + 1 <= r.ny - 1, okz = z + 1 <= r.nz - 1;
      uint32_t a = 0, as = 0, b = 0, bs = 0, c = 0, cs = 0, e = 0, es = 0;
      if (valid) {
        const uint32_t* R0 = brow(bits, r, y, z);  // bit row (y + dy, z + dz) = R0 + (dz * BY + dy) * W
        const long long BW = (long long)r.BY * W;
        const long long wrow = r.wpre0 + (g - r.row0) * (long long)W;  // word prefixes of row (y, z)
        const long long WZ = (long long)(r.ny + 1) * W;
        const bool nx1 = w + 1 < W;
        a = R0[w]; b = R0[W + w]; c = R0[BW + w]; e = R0[BW + W + w];
        const uint32_t an = nx1 ? R0[w + 1] : 0u, bn = nx1 ? R0[W + w + 1] : 0u;
        const uint32_t cn = nx1 ? R0[BW + w + 1] : 0u, en2 = nx1 ? R0[BW + W + w + 1] : 0u;
        as = shift1(a, an); bs = shift1(b, bn); cs = shift1(c, cn); es = shift1(e, en2);
        const uint32_t f = R0[2 * W + w], gg = R0[2 * BW + w], h = R0[BW + 2 * W + w], i2 = R0[2 * BW + W + w];
        S.own[0][lane] = make_int4((int)(a ^ as), (int)(a ^ b), (int)(a ^ c), wpre[wrow + w]);
        S.own[1][lane] = make_int4((int)(b ^ bs), (int)(b ^ f), (int)(b ^ e), oky ? wpre[wrow + W + w] : 0);
        S.own[2][lane] = make_int4((int)(c ^ cs), (int)(c ^ e), (int)(c ^ gg), okz ? wpre[wrow + WZ + w] : 0);
        S.own[3][lane] =
            make_int4((int)(e ^ es), (int)(e ^ h), (int)(e ^ i2), oky && okz ? wpre[wrow + WZ + W + w] : 0);
        // next word, bit 0: crossings along x and y of the owner rows, and their prefixes
        int o0 = 0, o1 = 0, o2 = 0, o3 = 0;
        if (nx1) {
          const uint32_t fn = R0[2 * W + w + 1], hn = R0[BW + 2 * W + w + 1];
          o0 = (wpre[wrow + w + 1] << 2) | (int)((((an ^ bn) & 1u) << 1) | ((an ^ (an >> 1)) & 1u));
          o1 = ((oky ? wpre[wrow + W + w + 1] : 0) << 2) | (int)((((bn ^ fn) & 1u) << 1) | ((bn ^ (bn >> 1)) & 1u));
          o2 = ((okz ? wpre[wrow + WZ + w + 1] : 0) << 2) | (int)((((cn ^ en2) & 1u) << 1) | ((cn ^ (cn >> 1)) & 1u));
          o3 = ((oky && okz ? wpre[wrow + WZ + W + w + 1] : 0) << 2) |
               (int)((((en2 ^ hn) & 1u) << 1) | ((en2 ^ (en2 >> 1)) & 1u));
        }
        S.onx[0][lane] = o0; S.onx[1][lane] = o1; S.onx[2][lane] = o2; S.onx[3][lane] = o3;
        S.vb[0][lane] = (int)row_base(prefix, g, 0);
        S.vb[1][lane] = oky ? (int)row_base(prefix, g + 1, 0) : 0;
        S.vb[2][lane] = okz ? (int)row_base(prefix, g + r.ny + 1, 0) : 0;
        S.vb[3][lane] = oky && okz ? (int)row_base(prefix, g + r.ny + 2, 0) : 0;
        S.tb[lane] = row_base(prefix, g, 1) + (w == 0 ? 0 : tpre[wrow + w]);
        u = (a ^ as) | (a ^ b) | (a ^ c);
        act = (a | as | b | bs | c | cs | e | es) & ~(a & as & b & bs & c & cs & e & es);
        m1v = w == 0 && (a & 1u);
        case_m1 = w == 0 ? (int)(((a & 1u) << 1) | ((b & 1u) << 3) | ((c & 1u) << 5) | ((e & 1u) << 7)) : 0;
      }
      S.cw[0][lane] = a; S.cw[1][lane] = as; S.cw[2][lane] = b; S.cw[3][lane] = bs;
      S.cw[4][lane] = c; S.cw[5][lane] = cs; S.cw[6][lane] = e; S.cw[7][lane] = es;
      S.y[lane] = y; S.z[lane] = z; S.wd[lane] = w; S.roi[lane] = roi; S.tab[lane] = r.tab; S.tcar[lane] = 0;
    }
    {
      const int t0 = __shfl_sync(0xffffffffu, S.roi[0], 0);  // lane 0's entry is always valid
      if (t0 != tag) {
        flush();
        tag = t0;
        since = 0;
      }
    }

    // ---- vertices: the x = -1 vertex opens word 0, then the positions by x --------
    {
      const int pc = __popc(u) + (m1v ? 1 : 0);
      const int pin = warp_incl(pc, lane);
      const int ptot = __shfl_sync(0xffffffffu, pin, 31);
      int o = pin - pc;
      if (m1v) S.list[o++] = (unsigned short)((lane << 6) | 32);
      for (uint32_t m = u; m; m &= m - 1) S.list[o++] = (unsigned short)((lane << 6) | (__ffs(m) - 1));
      __syncwarp();
      for (int j = lane; j < ptot; j += 32) {
        const unsigned short en = S.list[j];
        const int src = en >> 6, bit = en & 63;
        const int16_t qy = (int16_t)(2 * S.y[src]), qz = (int16_t)(2 * S.z[src]);
        long long id = S.vb[0][src];
        if (bit == 32) {
          if (id < vcap) {
            idx2[3 * id] = (int16_t)(-1); idx2[3 * id + 1] = qy; idx2[3 * id + 2] = qz;
          } else {
            err |= DEV_ERR_VCAP;
          }
          continue;
        }
        const int4 o0 = S.own[0][src];
        const uint32_t ex = (uint32_t)o0.x, ey = (uint32_t)o0.y, ez = (uint32_t)o0.z, low = (1u << bit) - 1u;
        id += o0.w + __popc(ex & low) + __popc(ey & low) + __popc(ez & low);
        const int16_t qx = (int16_t)(2 * (32 * S.wd[src] + bit));
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          if (!((((ax == 0 ? ex : (ax == 1 ? ey : ez)) >> bit) & 1u))) continue;
          if (id < vcap) {
            idx2[3 * id] = (int16_t)(qx + (ax == 0));
            idx2[3 * id + 1] = (int16_t)(qy + (ax == 1));
            idx2[3 * id + 2] = (int16_t)(qz + (ax == 2));
          } else {
            err |= DEV_ERR_VCAP;
          }
          ++id;
        }
      }
      __syncwarp();
    }

    // ---- active cubes: triangles, volume and case counts ---------------------------
    const int cc = __popc(act) + (case_m1 ? 1 : 0);
    const int cin = warp_incl(cc, lane);
    const int ctot = __shfl_sync(0xffffffffu, cin, 31);
    if (ctot == 0) continue;  // warp-uniform
    if (since + (unsigned int)ctot > 65535u) {  // no count can pass 16 bits
      flush();
      since = 0;
    }
    since += (unsigned int)ctot;
    {
      int o = cin - cc;
      if (case_m1) S.list[o++] = (unsigned short)((lane << 6) | 32);
      for (uint32_t m = act; m; m &= m - 1) S.list[o++] = (unsigned short)((lane << 6) | (__ffs(m) - 1));
    }
    __syncwarp();
    for (int j0 = 0; j0 < ctot; j0 += 32) {
      const int j = j0 + lane;
      const bool on = j < ctot;
      int src = -1, bit = 0, cs = 0, ntri = 0, roi = -1;
      const BinCase* bc = nullptr;
      if (on) {
        const unsigned short en = S.list[j];
        src = en >> 6;
        bit = en & 63;
        const int bq = bit == 32 ? 0 : bit;
        const uint32_t k0w = S.cw[0][src] >> bq, k1 = S.cw[1][src] >> bq, k2 = S.cw[2][src] >> bq,
                       k3 = S.cw[3][src] >> bq, k4 = S.cw[4][src] >> bq, k5 = S.cw[5][src] >> bq,
                       k6 = S.cw[6][src] >> bq, k7 = S.cw[7][src] >> bq;
        cs = bit == 32 ? (int)(((k0w & 1u) << 1) | ((k2 & 1u) << 3) | ((k4 & 1u) << 5) | ((k6 & 1u) << 7))
                       : (int)((k0w & 1u) | ((k1 & 1u) << 1) | ((k2 & 1u) << 2) | ((k3 & 1u) << 3) |
                               ((k4 & 1u) << 4) | ((k5 & 1u) << 5) | ((k6 & 1u) << 6) | ((k7 & 1u) << 7));
        roi = S.roi[src];
        bc = &tab[S.tab[src] * 256 + cs];
        ntri = bc->ntri;
        // owner-row prefixes and crossings at x (cx = 0) and x + 1 (cx = 1)
        int p0[4], p1[4];
        unsigned int x0[4], y0[4], x1[4], y1[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int4 ow = S.own[kk][src];
          const uint32_t ex = (uint32_t)ow.x, ey = (uint32_t)ow.y, ez = (uint32_t)ow.z;
          if (bit == 32) {  // x = -1: the row's first vertex; x + 1 = 0: bit 0 of word 0
            p0[kk] = 0; x0[kk] = 0u; y0[kk] = 0u;
            p1[kk] = ow.w; x1[kk] = ex & 1u; y1[kk] = ey & 1u;
          } else {
            const uint32_t low = (1u << bit) - 1u;
            p0[kk] = ow.w + __popc(ex & low) + __popc(ey & low) + __popc(ez & low);
            x0[kk] = (ex >> bit) & 1u; y0[kk] = (ey >> bit) & 1u;
            if (bit == 31) {
              const int nx = S.onx[kk][src];
              p1[kk] = nx >> 2; x1[kk] = (unsigned int)(nx & 1); y1[kk] = (unsigned int)((nx >> 1) & 1);
            } else {
              p1[kk] = p0[kk] + (int)(x0[kk] + y0[kk] + ((ez >> bit) & 1u));
              x1[kk] = (ex >> (bit + 1)) & 1u; y1[kk] = (ey >> (bit + 1)) & 1u;
            }
          }
        }
#pragma unroll
        for (int ed = 0; ed < 12; ++ed) {
          const int corner = (int)((kEdgeCorner >> (3 * ed)) & 7ull), ax = (int)((kEdgeAxis >> (2 * ed)) & 3u);
          const int kk = ((corner >> 1) & 1) + 2 * (corner >> 2);
          const bool hi = corner & 1;
          int rank = hi ? p1[kk] : p0[kk];
          if (ax >= 1) rank += (int)(hi ? x1[kk] : x0[kk]);
          if (ax >= 2) rank += (int)(hi ? y1[kk] : y0[kk]);
          S.vid[ed][lane] = S.vb[kk][src] + rank;
        }
      }
      // triangle ids: the word's base + its triangles already written + the
      // triangles of the word's earlier cubes in this round (runs of equal src)
      const int tin = warp_incl(ntri, lane);
      const int tex = tin - ntri;
      const unsigned int peers = __match_any_sync(0xffffffffu, src);
      const int seg0 = __shfl_sync(0xffffffffu, tex, __ffs(peers) - 1);
      const int seglast = 31 - __clz(peers);
      long long vsum = 0;
      if (on) {
        const unsigned long long t4 = bc->tri4;
        long long tid = S.tb[src] + S.tcar[src] + (tex - seg0);
        for (int t = 0; t < ntri; ++t, ++tid) {
          const int e0 = (int)((t4 >> (12 * t)) & 15ull), e1 = (int)((t4 >> (12 * t + 4)) & 15ull),
                    e2 = (int)((t4 >> (12 * t + 8)) & 15ull);
          if (tid < tcap) {
            tri[3 * tid] = S.vid[e0][lane];
            tri[3 * tid + 1] = S.vid[e1][lane];
            tri[3 * tid + 2] = S.vid[e2][lane];
          } else {
            err |= DEV_ERR_TCAP;
          }
        }
        // exact volume in half-voxel units relative to the padded-box centre
        const Roi& r = rois[roi];
        const int x = bit == 32 ? -1 : 32 * S.wd[src] + bit;
        const long long ox = 2LL * x - (r.nx - 1), oy = 2LL * S.y[src] - (r.ny - 1),
                        oz = 2LL * S.z[src] - (r.nz - 1);
        vsum = ox * bc->nsum[0] + oy * bc->nsum[1] + oz * bc->nsum[2] + bc->tsum;
      }
      __syncwarp();  // every lane has read the carries
      if (on && lane == seglast) S.tcar[src] += tin - seg0;
      __syncwarp();
      // |vsum| of one cube < 5e6, so a warp's sum fits in 32 bits; cubes of
      // the tagged ROI are counted in the warp, others (a ROI boundary inside
      // the warp's words) go straight to global memory
      const unsigned int same_roi = __match_any_sync(0xffffffffu, roi);
      const int vs = __reduce_add_sync(same_roi, (int)vsum);
      if (roi >= 0 && lane == __ffs(same_roi) - 1 && vs) {
        if (roi == tag) vacc += vs;
        else atomicAdd((unsigned long long*)&out[roi].vsum, (unsigned long long)(long long)vs);
      }
      const long long key = roi >= 0 ? (long long)roi * 256 + cs : -1;
      const unsigned int same_case = __match_any_sync(0xffffffffu, key);
      if (roi >= 0 && lane == __ffs(same_case) - 1) {
        if (roi == tag) hist[cs] = (unsigned short)(hist[cs] + __popc(same_case));
        else atomicAdd(&case_hist[key], (unsigned long long)__popc(same_case));
      }
    }
    __syncwarp();
  }
  flush();
  if (err) atomicOr(&tot->status, err);
}

// Mask volume and area per ROI (one block per ROI, fixed order):
//   6V = det(diag(s / 2)) * vsum,  2A = sum over cases of count * area2 of the case.
__global__ void k_mask_totals(const Roi* rois, int n, const BinCase* tab,
                              const unsigned long long* case_hist, RoiOut* out) {
  pdl_enter();
  __shared__ double s[256];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const Roi& r = rois[i];
    double a = 0.0;
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
      const unsigned long long cnt = case_hist[(long long)i * 256 + c];
      if (cnt) a += (double)cnt * tab[r.tab * 256 + c].area2;
    }
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double h3 = (0.5 * r.sx) * (0.5 * r.sy) * (0.5 * r.sz);
      const double vol6 = (double)out[i].vsum * h3;
      out[i].vol6 = vol6;
      out[i].area2 = s[0];
      closed_form_features(vol6 / 6.0, s[0] * 0.5, out[i].derived);
      out[i].has_derived = 1;
    }
    __syncthreads();
  }
}

// ---- voxel-coordinate moments -------------------------------------------------------
// Exact integer moments of the inside voxels' index coordinates per ROI (for
// the principal axes of the Shape class): every bitset word contributes
// through popcounts of its bit-index planes (sum of set bit positions b and of
// b^2), combined with the word's x0 = 32 w and its row (y, z).  One thread
// per word over contiguous per-block ranges (like the packing pass); a
// thread's sums stay in registers while its ROI is the same, a block adds its
// own ROI's sums with one atomic per moment.
// Exact index-coordinate moments of the inside voxels, one thread per voxel
// row (y, z) of a ROI: the row's count c, sum x and sum x^2 come from the
// packed words (popcounts against the bit-position planes), and the row adds
// c, y c, z c, ... to the ROI's nine sums.  Warps whose rows share one ROI
// reduce by shuffles first; a block's first ROI collects in shared memory.
__global__ void k_moments(const uint32_t* bits, const Roi* rois, int n, long long rows, RoiOut* out,
                          MeshTotals* tot) {
  pdl_enter();
  __shared__ unsigned long long s_m[9];
  __shared__ bool s_last;
  if (threadIdx.x < 9) s_m[threadIdx.x] = 0ull;
  const long long blk0 = (long long)blockIdx.x * blockDim.x;
  const int block_roi = blk0 < rows ? (n == 1 ? 0 : roi_of_row(rois, n, blk0)) : -1;
  __syncthreads();
  for (long long base = blk0; base < rows; base += (long long)gridDim.x * blockDim.x) {
    const long long g = base + threadIdx.x;
    unsigned long long m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = 0ull;
    int ri = -1;
    if (g < rows) {
      ri = n == 1 ? 0 : roi_of_row(rois, n, g);
      const Roi& r = rois[ri];
      const long long local = g - r.row0;
      const unsigned long long zz = (unsigned long long)(local / (r.ny + 1));
      const unsigned long long yy = (unsigned long long)(local - (long long)zz * (r.ny + 1));
      if (yy < (unsigned long long)r.ny && zz < (unsigned long long)r.nz) {
        const uint32_t* row = bits + r.word0 + ((long long)(zz + 1) * r.BY + (long long)(yy + 1)) * r.W;
        const uint32_t M[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
        unsigned long long c = 0, sx = 0, sxx = 0;
        for (int w = 0; w < r.W; ++w) {
          const uint32_t B = __ldcg(row + w);
          if (B == 0u) continue;
          unsigned int cw, sb, sbb;
          if (B == 0xFFFFFFFFu) {
            cw = 32; sb = 496; sbb = 10416;  // sums of b and b^2 over b = 0 .. 31
          } else {
            cw = __popc(B); sb = 0; sbb = 0;
#pragma unroll
            for (int k = 0; k < 5; ++k) {  // b = sum_k 2^k [bit k of b]
              const unsigned int pk = __popc(B & M[k]);
              sb += pk << k;
              sbb += pk << (2 * k);
#pragma unroll
              for (int l = k + 1; l < 5; ++l) sbb += __popc(B & M[k] & M[l]) << (k + l + 1);
            }
          }
          const unsigned long long x0 = 32ull * (unsigned long long)w;
          c += cw;
          sx += x0 * cw + sb;
          sxx += x0 * (x0 * cw + 2ull * sb) + sbb;
        }
        m[0] = sx; m[1] = yy * c; m[2] = zz * c;
        m[3] = sxx; m[4] = yy * yy * c; m[5] = zz * zz * c;
        m[6] = yy * sx; m[7] = zz * sx; m[8] = yy * zz * c;
      }
    }
    const int r0 = __shfl_sync(0xffffffffu, ri, 0);
    const bool uniform = __all_sync(0xffffffffu, ri == r0 || ri < 0);
    if (uniform) {
      for (int k = 0; k < 9; ++k) {
        unsigned long long v = m[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        m[k] = v;
      }
      if ((threadIdx.x & 31) == 0 && r0 >= 0) {
        for (int k = 0; k < 9; ++k)
          if (m[k]) {
            if (r0 == block_roi) atomicAdd(&s_m[k], m[k]);
            else atomicAdd(&out[r0].mom[k], m[k]);
          }
      }
    } else if (ri >= 0) {  // a warp across a ROI boundary (batches)
      for (int k = 0; k < 9; ++k)
        if (m[k]) atomicAdd(&out[ri].mom[k], m[k]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 9 && block_roi >= 0 && s_m[threadIdx.x]) atomicAdd(&out[block_roi].mom[threadIdx.x], s_m[threadIdx.x]);
  // the block that finishes last: principal axes of every ROI (FP64, one
  // thread per ROI; beside the emit pass, off the critical path)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tot->mom_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    unsigned long long mom[9];
    for (int k = 0; k < 9; ++k) mom[k] = __ldcg(&out[i].mom[k]);
    principal_axes(__ldcg(&out[i].nvox), mom, rois[i].sx, rois[i].sy, rois[i].sz, out[i].derived);
  }
}

// Lanes per row: several words per lane, so the per-row work (ROI lookup,
// row addresses, scans) is shared by more words -- four for narrow rows (crop
// batches), two for wide ones (the emit list then keeps fewer rows per warp).
int group_lanes(int W) {
  const int per = W <= 8 ? 4 : 2;
  int L = 1;
  while (per * L < W && L < 32) L <<= 1;
  return L;
}

}  // namespace

// ---- host ---------------------------------------------------------------------------

namespace {
// Case tables built so far, per (device, spacing), for the life of the
// process: a new workspace or batch with a known spacing copies its table
// instead of rebuilding it.  The buffers are never freed (one 256-case table
// per distinct spacing); a device reset invalidates them.
struct TableCache {
  std::mutex mu;
  std::map<std::array<double, 4>, const BinCase*> tabs;  // key: device, sx, sy, sz
};
TableCache& table_cache() {
  static TableCache* c = new TableCache;  // never destroyed: no teardown order issues at exit
  return *c;
}
}  // namespace

rad_status mesh_tables(const double* spacings_host, int n_tabs, MeshScratch& s, cudaStream_t st) {
  RAD_TRY(s.bintab.reserve(sizeof(BinCase) * 256 * std::max(n_tabs, 1)));
  RAD_TRY(s.tabsp.reserve(sizeof(double) * 3 * std::max(n_tabs, 1)));
  int dev = 0;
  RAD_CUDA(cudaGetDevice(&dev));
  TableCache& tc = table_cache();
  std::lock_guard<std::mutex> lock(tc.mu);
  auto key = [&](int k) {
    return std::array<double, 4>{(double)dev, spacings_host[3 * k], spacings_host[3 * k + 1], spacings_host[3 * k + 2]};
  };
  std::vector<double> miss;
  std::vector<int> miss_k;
  for (int k = 0; k < n_tabs; ++k)
    if (!tc.tabs.count(key(k))) {
      miss.insert(miss.end(), {spacings_host[3 * k], spacings_host[3 * k + 1], spacings_host[3 * k + 2]});
      miss_k.push_back(k);
    }
  if (!miss_k.empty()) {  // build the new ones in one launch, and finish before publishing them
    BinCase* fresh = nullptr;
    RAD_CUDA(cudaMalloc(&fresh, sizeof(BinCase) * 256 * miss_k.size()));
    RAD_CUDA(cudaMemcpyAsync(s.tabsp.p, miss.data(), sizeof(double) * miss.size(), cudaMemcpyHostToDevice, st));
    RAD_LAUNCH("mc_binary_table", k_binary_table, (int)miss_k.size(), 256, 0, st, s.tabsp.as<double>(), fresh);
    RAD_CUDA(cudaStreamSynchronize(st));
    for (size_t m = 0; m < miss_k.size(); ++m) tc.tabs[key(miss_k[m])] = fresh + 256 * m;
  }
  for (int k = 0; k < n_tabs; ++k)
    RAD_CUDA(cudaMemcpyAsync(s.bintab.as<BinCase>() + 256 * k, tc.tabs[key(k)], sizeof(BinCase) * 256,
                             cudaMemcpyDeviceToDevice, st));
  return RAD_OK;
}

rad_status mesh_count(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, cudaStream_t st) {
  const long long nchunks = (b.rows + kScanChunk - 1) / kScanChunk;
  RAD_TRY(s.bits.reserve(sizeof(uint32_t) * b.words));
  RAD_TRY(s.counts.reserve(sizeof(int4) * b.rows));
  RAD_TRY(s.wpre.reserve(sizeof(int) * b.wpre));
  RAD_TRY(s.tpre.reserve(sizeof(int) * b.wpre));
  RAD_TRY(s.wlist.reserve(sizeof(int2) * b.wpre));
  RAD_TRY(s.prefix.reserve(sizeof(long long) * 4 * b.rows));
  const size_t tiles_bytes = sizeof(ScanTile<4>) * nchunks, scan_bytes = tiles_bytes + 2 * sizeof(unsigned int);
  RAD_TRY(s.chunk.reserve(scan_bytes));  // look-back state of the row scan and its two tickets
  RAD_TRY(s.hist.reserve(sizeof(unsigned long long) * 256 * b.n));
  RAD_TRY(s.partial.reserve(sizeof(double) * 2 * num_sms() * kCubeBlocksPerSM));
  ZeroSet zs{};
  zero_add(zs, tot, sizeof(MeshTotals));
  zero_add(zs, out, sizeof(RoiOut) * b.n);
  zero_add(zs, s.hist.p, sizeof(unsigned long long) * 256 * b.n);
  zero_add(zs, s.chunk.p, scan_bytes);
  const int sms = num_sms();
  const int pack_blocks = wave_grid(k_pack<false>, 256, (b.words + 255) / 256);
  if (b.soft)
    RAD_LAUNCH("mc_pack_f32", k_pack<true>, pack_blocks, 256, 0, st, b.rois, b.n, b.words, s.bits.as<uint32_t>(), zs);
  else
    RAD_LAUNCH("mc_pack_u8", k_pack<false>, pack_blocks, 256, 0, st, b.rois, b.n, b.words, s.bits.as<uint32_t>(), zs);
  const long long warps_needed = (b.rows + (32 / b.L) - 1) / (32 / b.L);
  const int rblocks = wave_grid(k_count, kCountThreads, (warps_needed + 7) / 8);
  RAD_LAUNCH("mc_count", k_count, rblocks, kCountThreads, 0, st, s.bits.as<uint32_t>(), b.rois, b.n, b.rows, b.L, b.Wc,
             s.counts.as<int4>(), s.wpre.as<int>(), s.tpre.as<int>(), s.wlist.as<int2>(), b.wpre, tot);
  RAD_LAUNCH("mc_scan_rows", k_scan_rows, (int)nchunks, 256, 0, st, s.counts.as<int4>(), b.rows, (int)nchunks,
             s.prefix.as<long long>(), s.chunk.as<ScanTile<4>>(), (unsigned int*)(s.chunk.as<char>() + tiles_bytes),
             tot, b.rois, b.n, out);
  return RAD_OK;
}

rad_status mesh_emit(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, int16_t* idx2, double* vt,
                     int32_t* tri, long long vcap, long long tcap, cudaStream_t st, bool totals) {
  // every active cube has at least one triangle: the cube list fits in tcap
  const long long ccap = std::max<long long>(tcap, 1);
  if (b.soft) RAD_TRY(s.cubes.reserve(sizeof(int4) * ccap));
  const int sms = num_sms();
  const long long warps_needed = (b.rows + (32 / b.L) - 1) / (32 / b.L);
  const int rblocks = (int)std::max<long long>(1, std::min<long long>((warps_needed + 7) / 8, (long long)sms * 8));
  // a whole number of blocks per SM: the 32-cube groups are dealt round-robin
  // over the blocks, so every SM gets the same number of groups (the FP64
  // pipes bound this kernel; a grid that is not a multiple of the SM count
  // leaves some SMs with twice the work of others)
  const int cblocks = sms * kCubeBlocksPerSM;
  if (b.soft) {
    RAD_LAUNCH("mc_rows_soft", k_rows<true>, rblocks, 256, 0, st, s.bits.as<uint32_t>(), b.rois, b.n, b.rows, b.L,
               b.Wc, s.counts.as<int4>(), s.wpre.as<int>(), s.prefix.as<long long>(), idx2,
               vt, s.cubes.as<int4>(), vcap, ccap, tot);
    RAD_LAUNCH("mc_cubes_soft", k_cubes<true>, cblocks, kCubeThreads, 0, st, s.bits.as<uint32_t>(), b.rois, b.n,
               s.wpre.as<int>(), s.prefix.as<long long>(), s.cubes.as<int4>(),
               (const BinCase*)nullptr, tri, ccap, tcap, tot, out, s.hist.as<unsigned long long>(),
               s.partial.as<double>());
  } else {
    // persistent: the list length is known on the device only; the words of
    // all rows bound it (a small mask launches a few blocks)
    const int eblocks = (int)std::max<long long>(
        1, std::min<long long>((long long)sms * kEmitBlocksPerSM, (b.wpre + 32 * kEmitWarps - 1) / (32 * kEmitWarps)));
    RAD_LAUNCH("mc_emit", k_emit, eblocks, kEmitThreads, 0, st, s.bits.as<uint32_t>(), b.rois, b.n,
               s.wlist.as<int2>(), b.wpre, s.wpre.as<int>(), s.tpre.as<int>(), s.prefix.as<long long>(),
               s.bintab.as<BinCase>(), idx2, tri, vcap, tcap, tot, out,
               s.hist.as<unsigned long long>());
    if (totals) RAD_TRY(mesh_totals(b, s, out, st));
  }
  return RAD_OK;
}

rad_status mesh_moments(const MeshBatch& b, MeshScratch& s, MeshTotals* tot, RoiOut* out, cudaStream_t st) {
  RAD_LAUNCH("mc_moments", k_moments, wave_grid(k_moments, 256, (b.rows + 255) / 256), 256, 0, st,
             s.bits.as<uint32_t>(), b.rois, b.n, b.rows, out, tot);
  return RAD_OK;
}

rad_status mesh_totals(const MeshBatch& b, MeshScratch& s, RoiOut* out, cudaStream_t st) {
  if (b.soft) return RAD_OK;  // the soft cube kernel finishes its own totals
  RAD_LAUNCH("mc_mask_totals", k_mask_totals, std::min(b.n, num_sms() * 8), 256, 0, st, b.rois, b.n,
             s.bintab.as<BinCase>(), s.hist.as<unsigned long long>(), out);
  return RAD_OK;
}

// Host description of a batch: ROI table entries, offsets and the group shape.
void plan_batch(const int64_t* dims, const void* const* data, const int* tab, const double* spacing, int n, bool soft,
                std::vector<Roi>& rois, MeshBatch& b) {
  rois.resize(n);
  long long rows = 0, words = 0, wpre = 0;
  int maxW = 1;
  for (int i = 0; i < n; ++i) {
    Roi& r = rois[i];
    r.data = data[i];
    r.nx = (int)dims[3 * i];
    r.ny = (int)dims[3 * i + 1];
    r.nz = (int)dims[3 * i + 2];
    r.W = (r.nx + 31) / 32;
    r.BY = r.ny + 3;
    r.BZ = r.nz + 3;
    r.vec16 = soft ? ((r.nx % 4) == 0 && (((uintptr_t)r.data) & 15) == 0)
                   : ((r.nx % 16) == 0 && (((uintptr_t)r.data) & 15) == 0);
    r.tab = tab ? tab[i] : 0;
    r.R = (long long)(r.ny + 1) * (r.nz + 1);
    r.row0 = rows;
    r.word0 = words;
    r.wpre0 = wpre;
    r.sx = spacing[3 * i];
    r.sy = spacing[3 * i + 1];
    r.sz = spacing[3 * i + 2];
    rows += r.R;
    words += (long long)r.BY * r.BZ * r.W;
    wpre += r.R * r.W;
    maxW = std::max(maxW, r.W);
  }
  b.n = n;
  b.soft = soft;
  b.rows = rows;
  b.words = words;
  b.wpre = wpre;
  b.L = group_lanes(maxW);
  b.Wc = ((maxW + b.L - 1) / b.L) * b.L;
}

}  // namespace rad
