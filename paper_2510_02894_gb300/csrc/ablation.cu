// FP64 all-pairs diameter kernels for the accumulation-pattern ablation
// (paper Sec. 3, "Optimization research and results", steps (1)-(4), and
// Fig. 3): the same exhaustive FP64 search over every vertex pair, with the
// running maxima kept four different ways.
//
//   (1) equal load: every thread takes an equal run of the linearised pair
//       index space (i < j), reads both vertices from global memory, and
//       pushes each improvement on the maximum it last saw straight into the
//       global result with an atomic;
//   (2) block atomics: as (1), but improvements go to a per-block result in
//       shared memory, and each block makes one global atomic at the end;
//   (3) shared-memory 2D structures: blocks take tile pairs; the B tile is
//       staged in shared memory as a [vertex][coordinate] array, and
//       improvements go to the block result in shared memory as in (2);
//   (4) thread-local accumulators: as (3), but every thread keeps its maxima
//       in registers and merges them once, through warp shuffles and shared
//       memory, into one global atomic per block.
//
// Step (5) (1D arrays instead of 2D structures, thread-local maxima, one
// partial per block and a final pass) is the plain FP64 kernel of the
// diameter engine (diam.cu).  Every variant evaluates the pinned FP64 d2 of
// every pair in the same order of operations, and all maxima use one total
// order: the larger d2, then the smaller (i, j).  So all five give identical
// results, bit for bit.
//
// The maximum of a category is a 128-bit key (Key128: the bits of d2, then
// ~(i << 32 | j)) updated with a 128-bit compare-and-swap loop.
#include "rad_internal.cuh"

namespace rad {
namespace {

// Category tests of a pair: 3D always; Slice, Column, Row when the two
// vertices share z, y, x (index-space positions, equal exactly when the
// doubled coordinates are equal).
__device__ __forceinline__ void offer(const double ui[3], const double uj[3], double d2, int i, int j,
                                      Key128* dst, Key128 seen[4]) {
  const Key128 k = make_key(d2, i, j);
  const bool in[4] = {true, ui[2] == uj[2], ui[1] == uj[1], ui[0] == uj[0]};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (in[q] && key_gt(k, seen[q])) seen[q] = atomic_max_key(&dst[q], k);
}

// First pair (i, j) of the linear index l over the rows i = 0 .. n-2 of the
// upper triangle (row i holds the n - 1 - i pairs (i, i+1 .. n-1)).
__device__ void pair_of_index(long long l, long long n, long long& i, long long& j) {
  // row start S(i) = i n - i (i + 1) / 2; the largest i with S(i) <= l
  const double b = 2.0 * (double)n - 1.0;
  long long r = (long long)((b - sqrt(b * b - 8.0 * (double)l)) * 0.5);
  r = max(0ll, min(r, n - 2));
  while (r > 0 && r * n - r * (r + 1) / 2 > l) --r;
  while (r + 1 <= n - 2 && (r + 1) * n - (r + 1) * (r + 2) / 2 <= l) ++r;
  i = r;
  j = l - (r * n - r * (r + 1) / 2) + r + 1;
}

// Variants (1) and (2): equal runs of the pair index space per thread.
template <bool kBlock>
__global__ void k_equal_load(const int16_t* idx2, const double* vt, long long n, double sx, double sy, double sz,
                             Key128* result) {
  __shared__ Key128 s_best[4];
  Key128* dst = result;
  if (kBlock) {
    if (threadIdx.x < 4) s_best[threadIdx.x] = Key128{0ull, 0ull};
    __syncthreads();
    dst = s_best;
  }
  const long long P = n * (n - 1) / 2;
  const long long T = (long long)gridDim.x * blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // [P t / T, P (t + 1) / T) without overflow for P up to 2^63 / 2^21
  const long long l0 = (long long)((__int128)P * t / T), l1 = (long long)((__int128)P * (t + 1) / T);
  Key128 seen[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) seen[q] = Key128{0ull, 0ull};
  if (l0 < l1) {
    long long i, j;
    pair_of_index(l0, n, i, j);
    double ui[3];
    vertex_u(idx2, vt, i, ui);
    for (long long l = l0; l < l1; ++l) {
      double uj[3];
      vertex_u(idx2, vt, j, uj);
      const double d2 = pin_d2(ui[0], ui[1], ui[2], uj[0], uj[1], uj[2], sx, sy, sz);
      offer(ui, uj, d2, (int)i, (int)j, dst, seen);
      if (++j == n) {
        ++i;
        j = i + 1;
        if (i < n) vertex_u(idx2, vt, i, ui);
      }
    }
  }
  if (kBlock) {
    __syncthreads();
    if (threadIdx.x < 4 && (s_best[threadIdx.x].hi | s_best[threadIdx.x].lo))
      atomic_max_key(&result[threadIdx.x], s_best[threadIdx.x]);
  }
}

constexpr int kTile = 256;

// Tile pair l of the upper triangle (ta <= tb).
__device__ __forceinline__ void tile_pair(long long l, long long& ta, long long& tb) {
  long long b = (long long)((sqrt(8.0 * (double)l + 1.0) - 1.0) * 0.5);
  while (b * (b + 1) / 2 > l) --b;
  while ((b + 1) * (b + 2) / 2 <= l) ++b;
  tb = b;
  ta = l - b * (b + 1) / 2;
}

// Variants (3) and (4): tile pairs per block, the B tile staged in shared
// memory as a [vertex][coordinate] array.
template <bool kLocal>
__global__ void __launch_bounds__(kTile) k_tiled_2d(const int16_t* idx2, const double* vt, long long n, double sx,
                                                   double sy, double sz, Key128* result) {
  __shared__ double sv[kTile][3];
  __shared__ Key128 s_best[4];
  __shared__ Key128 s_warp[4][kTile / 32];
  if (threadIdx.x < 4) s_best[threadIdx.x] = Key128{0ull, 0ull};
  const long long nt = (n + kTile - 1) / kTile;
  const long long npairs = nt * (nt + 1) / 2;
  Key128 seen[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) seen[q] = Key128{0ull, 0ull};
  for (long long l = blockIdx.x; l < npairs; l += gridDim.x) {
    long long ta, tb;
    tile_pair(l, ta, tb);
    const long long jb = tb * kTile;
    __syncthreads();
    if (jb + threadIdx.x < n) {
      double u[3];
      vertex_u(idx2, vt, jb + threadIdx.x, u);
      sv[threadIdx.x][0] = u[0];
      sv[threadIdx.x][1] = u[1];
      sv[threadIdx.x][2] = u[2];
    }
    __syncthreads();
    const long long i = ta * kTile + threadIdx.x;
    if (i >= n) continue;
    double ui[3];
    vertex_u(idx2, vt, i, ui);
    const int jend = (int)min((long long)kTile, n - jb);
    for (int jj = 0; jj < jend; ++jj) {
      const long long j = jb + jj;
      if (j <= i) continue;
      const double uj[3] = {sv[jj][0], sv[jj][1], sv[jj][2]};
      const double d2 = pin_d2(ui[0], ui[1], ui[2], uj[0], uj[1], uj[2], sx, sy, sz);
      if (kLocal) {
        const Key128 k = make_key(d2, (int)i, (int)j);
        const bool in[4] = {true, ui[2] == uj[2], ui[1] == uj[1], ui[0] == uj[0]};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (in[q] && key_gt(k, seen[q])) seen[q] = k;
      } else {
        offer(ui, uj, d2, (int)i, (int)j, s_best, seen);
      }
    }
  }
  if (kLocal) {  // thread maxima: warp shuffles, then one slot per warp
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Key128 k = seen[q];
      for (int off = 16; off > 0; off >>= 1) {
        Key128 o;
        o.lo = __shfl_xor_sync(0xffffffffu, k.lo, off);
        o.hi = __shfl_xor_sync(0xffffffffu, k.hi, off);
        if (key_gt(o, k)) k = o;
      }
      if (lane == 0) s_warp[q][wid] = k;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      Key128 k = s_warp[threadIdx.x][0];
      for (int w = 1; w < kTile / 32; ++w)
        if (key_gt(s_warp[threadIdx.x][w], k)) k = s_warp[threadIdx.x][w];
      s_best[threadIdx.x] = k;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && (s_best[threadIdx.x].hi | s_best[threadIdx.x].lo))
    atomic_max_key(&result[threadIdx.x], s_best[threadIdx.x]);
}

__global__ void k_keys_final(const Key128* keys, DiamResult* out) {
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    const Key128 k = keys[q];
    const bool ok = (k.hi | k.lo) != 0ull;
    const unsigned long long pr = ~k.lo;
    out->d2[q] = ok ? __longlong_as_double((long long)k.hi) : 0.0;
    out->i[q] = ok ? (int)(pr >> 32) : -1;
    out->j[q] = ok ? (int)(pr & 0xffffffffull) : -1;
  }
}

}  // namespace

rad_status diam_fp64_variant(int variant, const int16_t* idx2, const double* vt, long long nv, const MeshDims& d,
                             const double sp[3], DiamScratch& s, DiamResult* out_dev, cudaStream_t st) {
  if (variant == RAD_FP64_PLAIN_1D) return diam_plain_fp64(idx2, vt, nv, d, sp, s, out_dev, st);
  if (variant < RAD_FP64_EQUAL_LOAD || variant > RAD_FP64_THREAD_LOCAL) {
    set_error("unknown FP64 diameter variant");
    return RAD_ERR_INVALID_ARG;
  }
  if (nv > (1ll << 31) - 1) {
    set_error("too many vertices for the FP64 all-pairs variants");
    return RAD_ERR_INVALID_ARG;
  }
  RAD_TRY(s.plain_part.reserve(sizeof(Key128) * 4));
  Key128* keys = s.plain_part.as<Key128>();
  RAD_CUDA(cudaMemsetAsync(keys, 0, sizeof(Key128) * 4, st));
  const int sms = num_sms();
  switch (variant) {
    case RAD_FP64_EQUAL_LOAD:
      RAD_LAUNCH("fp64_equal_load", k_equal_load<false>, sms * 8, 256, 0, st, idx2, vt, nv, sp[0], sp[1], sp[2],
                 keys);
      break;
    case RAD_FP64_BLOCK_ATOMICS:
      RAD_LAUNCH("fp64_block_atomics", k_equal_load<true>, sms * 8, 256, 0, st, idx2, vt, nv, sp[0], sp[1], sp[2],
                 keys);
      break;
    case RAD_FP64_SHARED_2D:
      RAD_LAUNCH("fp64_shared_2d", k_tiled_2d<false>, sms * 4, kTile, 0, st, idx2, vt, nv, sp[0], sp[1], sp[2],
                 keys);
      break;
    default:
      RAD_LAUNCH("fp64_thread_local", k_tiled_2d<true>, sms * 4, kTile, 0, st, idx2, vt, nv, sp[0], sp[1], sp[2],
                 keys);
      break;
  }
  RAD_LAUNCH("fp64_keys_final", k_keys_final, 1, 32, 0, st, keys, out_dev);
  return RAD_OK;
}

}  // namespace rad
