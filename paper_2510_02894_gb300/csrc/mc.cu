// Marching cubes on a padded mask (paper Sec. 2, "Marching cubes fused
// parallel kernels"): every cube of the implicitly zero-padded grid is tested
// against the iso level, crossing edges become vertices, the cube's case
// selects its polygons, and the mesh volume and surface area are summed.
//
// GB300 layout of the pass:
//   k_pack   the mask (uint8 or float32) is read once, coalesced and
//            vectorised (16-byte loads), and packed to one bit per voxel
//            (32 voxels per word) with zero rows around it; the packed grid
//            is 1/8 (1/32) of the input and stays in L2 for the passes below.
//   k_count  one group of lanes per x-row (y, z): crossing-edge bits by XOR of
//            neighbouring rows, counted with popc; active cubes by OR/AND of
//            the four rows of a cube row; per-row vertex, triangle and voxel
//            counts.
//   k_scan_* chunked exclusive scan of the row counts (vertex and triangle
//            ids follow the canonical (z, y, x, axis) order).
//   k_emit   re-derives the bits of the 3 x 3 neighbouring rows, ranks every
//            crossing edge with popc + group scans, writes vertices and
//            triangles, and reduces 6V and 2A in FP64 with a fixed-order tree
//            (deterministic).
#include <stdio.h>

#include <algorithm>

#include "mc_tables.inc"
#include "rad_internal.cuh"

namespace rad {

namespace {

constexpr int kScanChunk = 2048;  // rows per scan chunk (256 threads x 8)
constexpr int kEmitBlocksPerSM = 4;
constexpr int kEmitThreads = 256;

__device__ __forceinline__ const uint32_t* brow(const uint32_t* bits, const MeshDims& d, int y, int z) {
  return bits + ((long long)(z + 1) * d.BY + (y + 1)) * d.W;
}

__device__ __forceinline__ uint32_t ldw(const uint32_t* row, int w, int W) { return w < W ? row[w] : 0u; }

// ---- pack ------------------------------------------------------------------------

__device__ __forceinline__ uint32_t nz4(uint32_t v) {
  // bit 7 of each byte set iff the byte is non-zero, gathered to 4 bits
  uint32_t t = (v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
  t = (t | v) & 0x80808080u;
  return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

__global__ void k_pack_u8(const uint8_t* __restrict__ mask, MeshDims d, bool vec16, uint32_t* __restrict__ bits) {
  long long total = (long long)d.BY * d.BZ * d.W;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int w = (int)(id % d.W);
    long long br = id / d.W;
    int y = (int)(br % d.BY) - 1, z = (int)(br / d.BY) - 1;
    uint32_t word = 0;
    if (y >= 0 && y < d.ny && z >= 0 && z < d.nz) {
      const uint8_t* row = mask + ((long long)z * d.ny + y) * d.nx;
      int x0 = w * 32;
      int n = min(32, d.nx - x0);
      if (vec16 && n == 32) {
        uint4 a = __ldg(reinterpret_cast<const uint4*>(row + x0));
        uint4 b = __ldg(reinterpret_cast<const uint4*>(row + x0 + 16));
        word = nz4(a.x) | (nz4(a.y) << 4) | (nz4(a.z) << 8) | (nz4(a.w) << 12) | (nz4(b.x) << 16) |
               (nz4(b.y) << 20) | (nz4(b.z) << 24) | (nz4(b.w) << 28);
      } else if (vec16 && n == 16) {
        uint4 a = __ldg(reinterpret_cast<const uint4*>(row + x0));
        word = nz4(a.x) | (nz4(a.y) << 4) | (nz4(a.z) << 8) | (nz4(a.w) << 12);
      } else {
        for (int i = 0; i < n; ++i) word |= (uint32_t)(row[x0 + i] != 0) << i;
      }
    }
    bits[id] = word;
  }
}

__global__ void k_pack_f32(const float* __restrict__ prob, MeshDims d, bool vec16, uint32_t* __restrict__ bits) {
  long long total = (long long)d.BY * d.BZ * d.W;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int w = (int)(id % d.W);
    long long br = id / d.W;
    int y = (int)(br % d.BY) - 1, z = (int)(br / d.BY) - 1;
    uint32_t word = 0;
    if (y >= 0 && y < d.ny && z >= 0 && z < d.nz) {
      const float* row = prob + ((long long)z * d.ny + y) * d.nx;
      int x0 = w * 32;
      int n = min(32, d.nx - x0);
      if (vec16 && (n & 3) == 0) {
        for (int i = 0; i < n; i += 4) {
          float4 v = __ldg(reinterpret_cast<const float4*>(row + x0 + i));
          word |= ((uint32_t)(v.x > 0.5f) << i) | ((uint32_t)(v.y > 0.5f) << (i + 1)) |
                  ((uint32_t)(v.z > 0.5f) << (i + 2)) | ((uint32_t)(v.w > 0.5f) << (i + 3));
        }
      } else {
        for (int i = 0; i < n; ++i) word |= (uint32_t)(row[x0 + i] > 0.5f) << i;
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

__global__ void k_count(const uint32_t* __restrict__ bits, MeshDims d, int L, int* __restrict__ counts) {
  const int lane = threadIdx.x & 31, sub = lane % L, gpw = 32 / L;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * gpw; base < d.R; base += nwarps * gpw) {
    long long item = base + lane / L;
    bool valid = item < d.R;
    int y = valid ? (int)(item % (d.ny + 1)) - 1 : -1;
    int z = valid ? (int)(item / (d.ny + 1)) - 1 : -1;
    const uint32_t* R00 = brow(bits, d, y, z);
    const uint32_t* R10 = brow(bits, d, y + 1, z);
    const uint32_t* R01 = brow(bits, d, y, z + 1);
    const uint32_t* R11 = brow(bits, d, y + 1, z + 1);
    int nv = 0, nt = 0, nvox = 0;
    for (int w = sub; w < d.W + ((L - d.W % L) % L); w += L) {
      uint32_t a = ldw(R00, w, d.W), an = ldw(R00, w + 1, d.W);
      uint32_t b = ldw(R10, w, d.W), bn = ldw(R10, w + 1, d.W);
      uint32_t c = ldw(R01, w, d.W), cn = ldw(R01, w + 1, d.W);
      uint32_t e = ldw(R11, w, d.W), en = ldw(R11, w + 1, d.W);
      uint32_t ex = a ^ shift1(a, an), ey = a ^ b, ez = a ^ c;
      nv += __popc(ex) + __popc(ey) + __popc(ez);
      if (y >= 0 && z >= 0) nvox += __popc(a);
      uint32_t as = shift1(a, an), bs = shift1(b, bn), cs = shift1(c, cn), es = shift1(e, en);
      uint32_t o = a | b | c | e | as | bs | cs | es;
      uint32_t n = a & b & c & e & as & bs & cs & es;
      uint32_t act = o & ~n;
      while (act) {
        int bit = __ffs(act) - 1;
        act &= act - 1;
        nt += MC_CASE_NTRI[cube_case(a, as, b, bs, c, cs, e, es, bit)];
      }
    }
    if (sub == 0) {
      // owner x = -1 (x-edge into voxel 0) and cube x = -1 (corners cx = 1 at x = 0)
      uint32_t a0 = ldw(R00, 0, d.W) & 1u, b0 = ldw(R10, 0, d.W) & 1u, c0 = ldw(R01, 0, d.W) & 1u,
               e0 = ldw(R11, 0, d.W) & 1u;
      nv += (int)a0;
      int cs = (int)((a0 << 1) | (b0 << 3) | (c0 << 5) | (e0 << 7));
      nt += MC_CASE_NTRI[cs];
    }
    for (int off = L / 2; off > 0; off >>= 1) {
      nv += __shfl_xor_sync(0xffffffffu, nv, off, L);
      nt += __shfl_xor_sync(0xffffffffu, nt, off, L);
      nvox += __shfl_xor_sync(0xffffffffu, nvox, off, L);
    }
    if (valid && sub == 0) {
      counts[3 * item] = nv;
      counts[3 * item + 1] = nt;
      counts[3 * item + 2] = nvox;
    }
  }
}

// ---- scan of row counts -------------------------------------------------------------

__global__ void k_scan_chunks(const int* __restrict__ counts, long long R, long long* __restrict__ prefix,
                              long long* __restrict__ chunk) {
  __shared__ long long sv[8], st[8], sx[8];
  const long long beg = (long long)blockIdx.x * kScanChunk;
  const int per = kScanChunk / 256;
  long long v[per], t[per];
  long long lv = 0, lt = 0, lx = 0;
  for (int i = 0; i < per; ++i) {
    long long r = beg + threadIdx.x * per + i;
    int cv = 0, ct = 0, cx = 0;
    if (r < R) { cv = counts[3 * r]; ct = counts[3 * r + 1]; cx = counts[3 * r + 2]; }
    v[i] = lv; t[i] = lt;
    lv += cv; lt += ct; lx += cx;
  }
  // block exclusive scan of (lv, lt); sum of lx
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long iv = lv, it = lt, ix = lx;
  for (int off = 1; off < 32; off <<= 1) {
    long long a = __shfl_up_sync(0xffffffffu, iv, off), b = __shfl_up_sync(0xffffffffu, it, off);
    if (lane >= off) { iv += a; it += b; }
  }
  for (int off = 16; off > 0; off >>= 1) ix += __shfl_xor_sync(0xffffffffu, ix, off);
  if (lane == 31) { sv[wid] = iv; st[wid] = it; }
  if (lane == 0) sx[wid] = ix;
  __syncthreads();
  long long wv = 0, wt = 0;
  for (int k = 0; k < wid; ++k) { wv += sv[k]; wt += st[k]; }
  long long ev = wv + iv - lv, et = wt + it - lt;
  for (int i = 0; i < per; ++i) {
    long long r = beg + threadIdx.x * per + i;
    if (r < R) { prefix[2 * r] = ev + v[i]; prefix[2 * r + 1] = et + t[i]; }
  }
  if (threadIdx.x == 255) {
    long long tx = 0;
    for (int k = 0; k < 8; ++k) tx += sx[k];
    chunk[3 * blockIdx.x] = ev + lv;
    chunk[3 * blockIdx.x + 1] = et + lt;
    chunk[3 * blockIdx.x + 2] = tx;
  }
}

// Single block: exclusive scan of the chunk totals in place; totals to *tot.
__global__ void k_scan_top(long long* __restrict__ chunk, int nchunks, MeshTotals* __restrict__ tot) {
  __shared__ long long sv[32], st[32], sx[32];
  long long carry_v = 0, carry_t = 0, carry_x = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < nchunks; base += blockDim.x) {
    const int c = base + threadIdx.x;
    long long v = 0, t = 0, x = 0;
    if (c < nchunks) { v = chunk[3 * c]; t = chunk[3 * c + 1]; x = chunk[3 * c + 2]; }
    long long iv = v, it = t, ix = x;
    for (int off = 1; off < 32; off <<= 1) {
      const long long a = __shfl_up_sync(0xffffffffu, iv, off), b = __shfl_up_sync(0xffffffffu, it, off);
      if (lane >= off) { iv += a; it += b; }
    }
    for (int off = 16; off > 0; off >>= 1) ix += __shfl_xor_sync(0xffffffffu, ix, off);
    if (lane == 31) { sv[wid] = iv; st[wid] = it; }
    if (lane == 0) sx[wid] = ix;
    __syncthreads();
    long long wv = 0, wt = 0, bv = 0, bt = 0, bx = 0;
    for (int k = 0; k < nw; ++k) {
      if (k < wid) { wv += sv[k]; wt += st[k]; }
      bv += sv[k]; bt += st[k]; bx += sx[k];
    }
    if (c < nchunks) {
      chunk[3 * c] = carry_v + wv + iv - v;
      chunk[3 * c + 1] = carry_t + wt + it - t;
    }
    carry_v += bv;
    carry_t += bt;
    carry_x += bx;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tot->nv = carry_v;
    tot->nt = carry_t;
    tot->nvox = carry_x;
  }
}

// ---- triangulation choice -----------------------------------------------------------
// Among a loop's admissible candidates (stored in ascending lexicographic order
// of their canonical triple lists): minimum area score, then maximum volume,
// then the first in list order.  Pinned FP64 arithmetic, so the same choice
// as any other implementation of the rule.
__device__ int select_candidate(int loop, const double (*w)[3], const double* sp) {
  const int k = MC_LOOP_K[loop], nt = k - 2;
  const int cb = MC_LOOP_CAND_BEGIN[loop], ce = MC_LOOP_CAND_BEGIN[loop + 1];
  if (ce - cb == 1) return cb;
  double sc[MC_MAX_CAND], vv[MC_MAX_CAND];
  double smin = 0.0;
  for (int c = cb; c < ce; ++c) {
    const int tb = MC_CAND_TRI_BEGIN[c];
    double s = 0.0, v = 0.0;
    for (int t = 0; t < nt; ++t) {
      const unsigned char* tr = &MC_CAND_TRIPLES[3 * (tb + t)];
      s = __dadd_rn(s, pin_tri_r(w[tr[0]], w[tr[1]], w[tr[2]]));
      v = __dadd_rn(v, pin_vol6(w[tr[0]], w[tr[1]], w[tr[2]]));
    }
    sc[c - cb] = s;
    vv[c - cb] = v;
    if (c == cb || s < smin) smin = s;
  }
  const double slim = __dadd_rn(smin, __dmul_rn(smin, 1e-12));
  double vmax = 0.0;
  bool have = false;
  for (int c = 0; c < ce - cb; ++c)
    if (sc[c] <= slim && (!have || vv[c] > vmax)) { vmax = vv[c]; have = true; }
  const double vlim = __dsub_rn(vmax, __dmul_rn(__dmul_rn(__dmul_rn(sp[0], sp[1]), sp[2]), 1e-9));
  for (int c = 0; c < ce - cb; ++c)
    if (sc[c] <= slim && vv[c] >= vlim) return cb + c;
  return cb;  // not reached
}

// Binary masks: every crossing sits at an edge midpoint, so the choice depends
// only on (case, spacing).  One thread per case writes MC_MAX_TRI triples.
__global__ void k_binary_table(double sx, double sy, double sz, unsigned char* __restrict__ tab) {
  const int cs = blockIdx.x * blockDim.x + threadIdx.x;
  if (cs >= 256) return;
  const double sp[3] = {sx, sy, sz};
  double w[12][3];
  for (int e = 0; e < 12; ++e) {
    const int c = MC_EDGE_CORNER[e], a = MC_EDGE_AXIS[e];
    for (int k = 0; k < 3; ++k)
      w[e][k] = __dmul_rn(__dadd_rn((double)((c >> k) & 1), k == a ? 0.5 : 0.0), sp[k]);
  }
  int n = 0;
  for (int l = MC_CASE_LOOP_BEGIN[cs]; l < MC_CASE_LOOP_BEGIN[cs + 1]; ++l) {
    const int c = select_candidate(l, w, sp);
    const int tb = MC_CAND_TRI_BEGIN[c];
    for (int t = 0; t < MC_LOOP_K[l] - 2; ++t, ++n)
      for (int q = 0; q < 3; ++q) tab[(cs * MC_MAX_TRI + n) * 3 + q] = MC_CAND_TRIPLES[3 * (tb + t) + q];
  }
}

// ---- emit ----------------------------------------------------------------------------

struct OwnerRow {
  uint32_t ex, ey, ez;  // crossing bits of this word (owner x = 32 w + bit)
  int cnt;              // crossings in this word
  long long pre;        // id of the first crossing of this word
  int exn, eyn;         // crossings at bit 0 of the next word (x-edge, y-edge)
};

__device__ __forceinline__ long long owner_rank(const OwnerRow& o, int bit, int a) {
  if (bit == 32) return o.pre + o.cnt + (a >= 1 ? o.exn : 0) + (a >= 2 ? o.eyn : 0);
  const uint32_t low = (1u << bit) - 1u;
  long long r = o.pre + __popc(o.ex & low) + __popc(o.ey & low) + __popc(o.ez & low);
  if (a >= 1) r += (o.ex >> bit) & 1u;
  if (a >= 2) r += (o.ey >> bit) & 1u;
  return r;
}

__device__ __forceinline__ float value_at(const float* p, const MeshDims& d, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0.0f;
  return __ldg(p + ((long long)z * d.ny + y) * d.nx + x);
}

__device__ __forceinline__ double crossing_t(double v0, double v1) {
  return __ddiv_rn(__dsub_rn(0.5, v0), __dsub_rn(v1, v0));
}

template <bool SOFT>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const uint32_t* __restrict__ bits, const float* __restrict__ prob,
                                                       MeshDims d, int L, double sx, double sy, double sz,
                                                       const long long* __restrict__ prefix,
                                                       const long long* __restrict__ chunk,
                                                       const unsigned char* __restrict__ bintab,
                                                       int16_t* __restrict__ idx2, double* __restrict__ vt,
                                                       int32_t* __restrict__ tri, long long vcap, long long tcap,
                                                       MeshTotals* __restrict__ tot, double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, sub = lane % L, gpw = 32 / L;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const double sp[3] = {sx, sy, sz};
  const double hs[3] = {0.5 * sx, 0.5 * sy, 0.5 * sz};
  const int nn[3] = {d.nx, d.ny, d.nz};
  double acc_v6 = 0.0, acc_a2 = 0.0;
  unsigned int err = 0;
  const int Wc = d.W + ((L - d.W % L) % L);  // word loop bound, uniform across groups

  for (long long base = warp * gpw; base < d.R; base += nwarps * gpw) {
    const long long item = base + lane / L;
    const bool valid = item < d.R;
    const int y = valid ? (int)(item % (d.ny + 1)) - 1 : -1;
    const int z = valid ? (int)(item / (d.ny + 1)) - 1 : -1;
    // bitset rows (y + dy, z + dz), dy, dz in 0..2
    const uint32_t* rows[3][3];
    for (int dz = 0; dz < 3; ++dz)
      for (int dy = 0; dy < 3; ++dy) rows[dz][dy] = brow(bits, d, y + dy, z + dz);
    // owner rows o = (oy, oz) in {0,1}^2: base vertex ids
    long long vb[2][2];
    bool orow_ok[2][2];
    for (int oz = 0; oz < 2; ++oz)
      for (int oy = 0; oy < 2; ++oy) {
        const bool ok = valid && (y + oy) <= d.ny - 1 && (z + oz) <= d.nz - 1;
        orow_ok[oz][oy] = ok;
        long long r = ok ? (long long)(z + oz + 1) * (d.ny + 1) + (y + oy + 1) : 0;
        vb[oz][oy] = ok ? prefix[2 * r] + chunk[3 * (r / kScanChunk)] : 0;
      }
    const long long tb = valid ? prefix[2 * item + 1] + chunk[3 * (item / kScanChunk) + 1] : 0;
    // ex_m1 of each owner row: x-edge from x = -1 into voxel 0
    int exm1[2][2];
    for (int oz = 0; oz < 2; ++oz)
      for (int oy = 0; oy < 2; ++oy) exm1[oz][oy] = (int)(ldw(rows[oz][oy], 0, d.W) & 1u);
    // cube x = -1: corners with cx = 1 are voxels x = 0
    const int case_m1 = (int)((exm1[0][0] << 1) | (exm1[0][1] << 3) | (exm1[1][0] << 5) | (exm1[1][1] << 7));
    const int ntri_m1 = MC_CASE_NTRI[case_m1];

    long long carry_o[2][2] = {{0, 0}, {0, 0}};
    long long carry_t = 0;
    for (int w = sub; w < Wc; w += L) {
      // words of the 8 rows needed, at w, w + 1, w + 2
      uint32_t m[3][3][3];
      for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
          for (int s = 0; s < 3; ++s)
            m[dz][dy][s] = (dz == 2 && dy == 2) ? 0u : ldw(rows[dz][dy], w + s, d.W);
      OwnerRow o[2][2];
      for (int oz = 0; oz < 2; ++oz)
        for (int oy = 0; oy < 2; ++oy) {
          const uint32_t a = m[oz][oy][0], an = m[oz][oy][1], ann = m[oz][oy][2];
          const uint32_t b = m[oz][oy + 1][0], bn = m[oz][oy + 1][1];
          const uint32_t c = m[oz + 1][oy][0];
          OwnerRow& r = o[oz][oy];
          r.ex = a ^ shift1(a, an);
          r.ey = a ^ b;
          r.ez = a ^ c;
          r.cnt = __popc(r.ex) + __popc(r.ey) + __popc(r.ez);
          r.exn = (int)((an ^ shift1(an, ann)) & 1u);
          r.eyn = (int)((an ^ bn) & 1u);
        }
      // group scans of the four owner-row counts and of the triangle counts
      const uint32_t A = m[0][0][0], An = m[0][0][1], B = m[0][1][0], Bn = m[0][1][1];
      const uint32_t C = m[1][0][0], Cn = m[1][0][1], E = m[1][1][0], En = m[1][1][1];
      const uint32_t As = shift1(A, An), Bs = shift1(B, Bn), Cs = shift1(C, Cn), Es = shift1(E, En);
      const uint32_t act = (A | B | C | E | As | Bs | Cs | Es) & ~(A & B & C & E & As & Bs & Cs & Es);
      int tcnt = 0;
      for (uint32_t a2 = act; a2; a2 &= a2 - 1) tcnt += MC_CASE_NTRI[cube_case(A, As, B, Bs, C, Cs, E, Es, __ffs(a2) - 1)];
      int incl[5] = {o[0][0].cnt, o[0][1].cnt, o[1][0].cnt, o[1][1].cnt, tcnt};
      const int own[5] = {incl[0], incl[1], incl[2], incl[3], incl[4]};
      for (int off = 1; off < L; off <<= 1)
        for (int q = 0; q < 5; ++q) {
          int v = __shfl_up_sync(0xffffffffu, incl[q], off, L);
          if (sub >= off) incl[q] += v;
        }
      int tot5[5];
      for (int q = 0; q < 5; ++q) tot5[q] = __shfl_sync(0xffffffffu, incl[q], L - 1, L);
      o[0][0].pre = carry_o[0][0] + exm1[0][0] + incl[0] - own[0];
      o[0][1].pre = carry_o[0][1] + exm1[0][1] + incl[1] - own[1];
      o[1][0].pre = carry_o[1][0] + exm1[1][0] + incl[2] - own[2];
      o[1][1].pre = carry_o[1][1] + exm1[1][1] + incl[3] - own[3];
      long long tpre = carry_t + ntri_m1 + incl[4] - own[4];

      if (valid && w < d.W) {
        // vertices owned by row (y, z), canonical order within the word
        if (orow_ok[0][0]) {
          long long id = vb[0][0] + o[0][0].pre;
          const OwnerRow& r = o[0][0];
          for (uint32_t u = r.ex | r.ey | r.ez; u; u &= u - 1) {
            const int bit = __ffs(u) - 1;
            const int x = w * 32 + bit;
            for (int a = 0; a < 3; ++a) {
              const uint32_t eb = a == 0 ? r.ex : (a == 1 ? r.ey : r.ez);
              if (!((eb >> bit) & 1u)) continue;
              if (id < vcap) {
                idx2[3 * id] = (int16_t)(2 * x + (a == 0));
                idx2[3 * id + 1] = (int16_t)(2 * y + (a == 1));
                idx2[3 * id + 2] = (int16_t)(2 * z + (a == 2));
                if (SOFT) {
                  double v0 = (double)value_at(prob, d, x, y, z);
                  double v1 = (double)value_at(prob, d, x + (a == 0), y + (a == 1), z + (a == 2));
                  vt[id] = crossing_t(v0, v1);
                }
              } else {
                err |= DEV_ERR_VCAP;
              }
              ++id;
            }
          }
          if (w == 0 && exm1[0][0]) {
            const long long id0 = vb[0][0];
            if (id0 < vcap) {
              idx2[3 * id0] = (int16_t)(-1);
              idx2[3 * id0 + 1] = (int16_t)(2 * y);
              idx2[3 * id0 + 2] = (int16_t)(2 * z);
              if (SOFT) vt[id0] = crossing_t(0.0, (double)value_at(prob, d, 0, y, z));
            } else {
              err |= DEV_ERR_VCAP;
            }
          }
        }
        // triangles of cube row (y, z): cube x = -1 first (lane of word 0), then ascending x
        long long tid = tb + tpre;
        int first_bit = (w == 0) ? -1 : 0;
        uint32_t cubes = act;
        for (int cb = first_bit; cb < 32; ++cb) {
          int cs;
          if (cb < 0) {
            if (!ntri_m1) continue;
            cs = case_m1;
            tid = tb;  // cube x = -1 comes first in the row
          } else {
            if (!((cubes >> cb) & 1u)) continue;
            cs = cube_case(A, As, B, Bs, C, Cs, E, Es, cb);
          }
          const int x = w * 32 + cb;  // cube lower corner x (may be -1)
          // vertex ids and positions of the cube's crossing edges
          const unsigned int emask = MC_CASE_EDGES[cs];
          long long vid[12];
          double P[12][3];
          double wl[12][3];
          for (int e = 0; e < 12; ++e) {
            if (!((emask >> e) & 1u)) continue;
            const int c = MC_EDGE_CORNER[e], a = MC_EDGE_AXIS[e];
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            const int ox = x + cx;
            long long r;
            if (ox < 0) r = 0;  // the x-edge of owner x = -1 is the row's first vertex
            else r = owner_rank(o[cz][cy], ox - w * 32, a);
            vid[e] = vb[cz][cy] + r;
            const int g[3] = {ox, y + cy, z + cz};
            double t = 0.5;
            if (SOFT) {
              const double v0 = (double)value_at(prob, d, g[0], g[1], g[2]);
              const double v1 = (double)value_at(prob, d, g[0] + (a == 0), g[1] + (a == 1), g[2] + (a == 2));
              t = crossing_t(v0, v1);
            }
            for (int k = 0; k < 3; ++k) {
              if (SOFT) {
                P[e][k] = ((double)g[k] - 0.5 * (double)(nn[k] - 1) + (k == a ? t : 0.0)) * sp[k];
                wl[e][k] = __dmul_rn(__dadd_rn((double)((c >> k) & 1), k == a ? t : 0.0), sp[k]);
              } else {
                P[e][k] = (double)(2 * g[k] + (k == a) - (nn[k] - 1)) * hs[k];
              }
            }
          }
          // triangles of the cube
          int nt = 0;
          unsigned char trs[MC_MAX_TRI][3];
          if (SOFT) {
            for (int l = MC_CASE_LOOP_BEGIN[cs]; l < MC_CASE_LOOP_BEGIN[cs + 1]; ++l) {
              const int cand = select_candidate(l, wl, sp);
              const int tb2 = MC_CAND_TRI_BEGIN[cand];
              for (int t = 0; t < MC_LOOP_K[l] - 2; ++t, ++nt)
                for (int q = 0; q < 3; ++q) trs[nt][q] = MC_CAND_TRIPLES[3 * (tb2 + t) + q];
            }
          } else {
            nt = MC_CASE_NTRI[cs];
            for (int t = 0; t < nt; ++t)
              for (int q = 0; q < 3; ++q) trs[t][q] = bintab[(cs * MC_MAX_TRI + t) * 3 + q];
          }
          for (int t = 0; t < nt; ++t, ++tid) {
            const int e0 = trs[t][0], e1 = trs[t][1], e2 = trs[t][2];
            if (tid < tcap) {
              tri[3 * tid] = (int32_t)vid[e0];
              tri[3 * tid + 1] = (int32_t)vid[e1];
              tri[3 * tid + 2] = (int32_t)vid[e2];
            } else {
              err |= DEV_ERR_TCAP;
            }
            const double* a = P[e0];
            const double* b = P[e1];
            const double* c = P[e2];
            acc_v6 += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                      a[2] * (b[0] * c[1] - b[1] * c[0]);
            const double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
            const double vx = c[0] - a[0], vy = c[1] - a[1], vz = c[2] - a[2];
            const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
            acc_a2 += sqrt(nx * nx + ny * ny + nz * nz);
          }
          if (cb < 0) tid = tb + tpre;  // resume at this lane's first cube of the word
        }
      }
      for (int oz = 0; oz < 2; ++oz)
        for (int oy = 0; oy < 2; ++oy) carry_o[oz][oy] += tot5[oz * 2 + oy];
      carry_t += tot5[4];
    }
  }
  // deterministic reduction: warp tree, then block, then the last CTA
  for (int off = 16; off > 0; off >>= 1) {
    acc_v6 += __shfl_xor_sync(0xffffffffu, acc_v6, off);
    acc_a2 += __shfl_xor_sync(0xffffffffu, acc_a2, off);
    err |= __shfl_xor_sync(0xffffffffu, err, off);
  }
  __shared__ double sv[kEmitThreads / 32], sa[kEmitThreads / 32];
  __shared__ unsigned int se[kEmitThreads / 32];
  __shared__ bool last;
  const int wid = threadIdx.x >> 5;
  if (lane == 0) { sv[wid] = acc_v6; sa[wid] = acc_a2; se[wid] = err; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = 0.0, ba = 0.0;
    unsigned int be = 0;
    for (int k = 0; k < kEmitThreads / 32; ++k) { bv += sv[k]; ba += sa[k]; be |= se[k]; }
    partial[2 * blockIdx.x] = bv;
    partial[2 * blockIdx.x + 1] = ba;
    if (be) atomicOr(&tot->status, be);
    __threadfence();
    const unsigned int ticket = atomicAdd(&tot->done_ctas, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double v = 0.0, a = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      v += __ldcg(&partial[2 * b]);
      a += __ldcg(&partial[2 * b + 1]);
    }
    tot->vol6 = v;
    tot->area2 = a;
    tot->done_ctas = 0;
  }
}

int group_lanes(int W) {
  int L = 1;
  while (L < W && L < 32) L <<= 1;
  return L;
}

}  // namespace

MeshDims make_dims(const int64_t dims[3]) {
  MeshDims d;
  d.nx = (int)dims[0];
  d.ny = (int)dims[1];
  d.nz = (int)dims[2];
  d.W = (d.nx + 31) / 32;
  d.BY = d.ny + 3;
  d.BZ = d.nz + 3;
  d.R = (long long)(d.ny + 1) * (d.nz + 1);
  return d;
}

rad_status mesh_count(const void* data, bool soft, const MeshDims& d, MeshScratch& s, MeshTotals* tot,
                      cudaStream_t st) {
  const long long words = (long long)d.BY * d.BZ * d.W;
  const long long nchunks = (d.R + kScanChunk - 1) / kScanChunk;
  RAD_TRY(s.bits.reserve(sizeof(uint32_t) * words));
  RAD_TRY(s.counts.reserve(sizeof(int) * 3 * d.R));
  RAD_TRY(s.prefix.reserve(sizeof(long long) * 2 * d.R));
  RAD_TRY(s.chunk.reserve(sizeof(long long) * 3 * nchunks));
  RAD_TRY(s.partial.reserve(sizeof(double) * 2 * num_sms() * kEmitBlocksPerSM));
  RAD_CUDA(cudaMemsetAsync(tot, 0, sizeof(MeshTotals), st));
  const int sms = num_sms();
  const bool vec16 = soft ? ((d.nx % 4) == 0 && (((uintptr_t)data) & 15) == 0)
                          : ((d.nx % 16) == 0 && (((uintptr_t)data) & 15) == 0);
  const int pack_blocks = (int)std::min<long long>((words + 255) / 256, (long long)sms * 16);
  if (soft)
    RAD_LAUNCH("mc_pack_f32", k_pack_f32, pack_blocks, 256, 0, st, (const float*)data, d, vec16,
               s.bits.as<uint32_t>());
  else
    RAD_LAUNCH("mc_pack_u8", k_pack_u8, pack_blocks, 256, 0, st, (const uint8_t*)data, d, vec16,
               s.bits.as<uint32_t>());
  const int L = group_lanes(d.W);
  const long long groups_needed = d.R;
  const long long warps_needed = (groups_needed + (32 / L) - 1) / (32 / L);
  const int cblocks = (int)std::max<long long>(1, std::min<long long>((warps_needed + 7) / 8, (long long)sms * 8));
  RAD_LAUNCH("mc_count", k_count, cblocks, 256, 0, st, s.bits.as<uint32_t>(), d, L, s.counts.as<int>());
  RAD_LAUNCH("mc_scan_chunks", k_scan_chunks, (int)nchunks, 256, 0, st, s.counts.as<int>(), d.R,
             s.prefix.as<long long>(), s.chunk.as<long long>());
  RAD_LAUNCH("mc_scan_top", k_scan_top, 1, 1024, 0, st, s.chunk.as<long long>(), (int)nchunks,
             tot);
  return RAD_OK;
}

rad_status mesh_emit(const void* data, bool soft, const MeshDims& d, const double sp[3], MeshScratch& s,
                     MeshTotals* tot, int16_t* idx2, double* vt, int32_t* tri, long long vcap, long long tcap,
                     cudaStream_t st) {
  if (!soft) {
    RAD_TRY(s.bintab.reserve(256 * MC_MAX_TRI * 3));
    if (!s.tab_valid || s.tab_spacing[0] != sp[0] || s.tab_spacing[1] != sp[1] || s.tab_spacing[2] != sp[2]) {
      RAD_LAUNCH("mc_binary_table", k_binary_table, 1, 256, 0, st, sp[0], sp[1], sp[2],
                 s.bintab.as<unsigned char>());
      s.tab_valid = true;
      for (int k = 0; k < 3; ++k) s.tab_spacing[k] = sp[k];
    }
  }
  const int L = group_lanes(d.W);
  const int blocks = num_sms() * kEmitBlocksPerSM;
  if (soft)
    RAD_LAUNCH("mc_emit_soft", k_emit<true>, blocks, kEmitThreads, 0, st, s.bits.as<uint32_t>(),
               (const float*)data, d, L, sp[0], sp[1], sp[2], s.prefix.as<long long>(), s.chunk.as<long long>(),
               (const unsigned char*)nullptr, idx2, vt, tri, vcap, tcap, tot,
               s.partial.as<double>());
  else
    RAD_LAUNCH("mc_emit", k_emit<false>, blocks, kEmitThreads, 0, st, s.bits.as<uint32_t>(), (const float*)nullptr,
               d, L, sp[0], sp[1], sp[2], s.prefix.as<long long>(), s.chunk.as<long long>(),
               s.bintab.as<unsigned char>(), idx2, vt, tri, vcap, tcap, tot,
               s.partial.as<double>());
  return RAD_OK;
}

}  // namespace rad
