// Diameters without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a framework owns
// the device memory budget (a caching allocator with a fixed pool, a
// real-time service that forbids allocation after start-up), or code that
// must not trigger the implicit synchronisation of cudaMalloc/cudaFree.
// rad_diameters_plain_fp64_noalloc serves them: the caller passes the
// vertices and the output buffers, and the only scratch this entry point
// uses is a file-scope static device array that the library image carries:
// it is resident on a device from the library module's load there until that
// device's context is destroyed.
//
// The kernel is a variant of the plain FP64 all-pairs diameter kernel: CTA c
// scans the 256-vertex tile rows c and T - 1 - c (T tile rows; row i holds
// the tiles j >= i), so every CTA covers about T + 1 tiles, and writes its
// best (d2, i, j) for 3D, Slice, Column and Row into slot c of the static
// array; a second kernel reduces the slots in fixed order into the caller's
// outputs.
#include <mutex>

#include "rad_internal.cuh"

namespace rad {
namespace {

constexpr int kNaTile = 256;
constexpr int kNaMaxTiles = 4096;  // 4096 tiles x 4 records x 16 B = 256 KB

struct NaBest {
  double d2;
  int i, j;
};

// Every call writes slots [0, tiles) before the reduction reads them, so the
// array needs no clearing between calls.
static __device__ __align__(256) NaBest g_na_scratch[kNaMaxTiles * 4];

__device__ __forceinline__ bool na_better(double d2, int i, int j, const NaBest& b) {
  if (b.i < 0) return i >= 0;
  if (i < 0) return false;
  if (d2 != b.d2) return d2 > b.d2;
  if (i != b.i) return i < b.i;
  return j < b.j;
}

__device__ __forceinline__ void na_take(NaBest& b, double d2, int i, int j) {
  if (na_better(d2, i, j, b)) { b.d2 = d2; b.i = i; b.j = j; }
}

// Tile row ti (tiles ti .. nt - 1) into the thread's maxima b; every thread
// of the block calls it (it synchronises the block).
__device__ void na_row(const int16_t* idx2, const double* vt, int n, int nt, int ti, double sx, double sy,
                       double sz, double (*su)[kNaTile], int (*sq)[kNaTile], NaBest b[4]) {
  const int i = ti * kNaTile + threadIdx.x;
  double ui[3] = {0.0, 0.0, 0.0};
  int qi[3] = {0, 0, 0};
  if (i < n) {
    vertex_u(idx2, vt, i, ui);
    for (int k = 0; k < 3; ++k) qi[k] = idx2[3 * i + k];
  }
  for (int tj = ti; tj < nt; ++tj) {
    const int jb = tj * kNaTile;
    __syncthreads();
    if (jb + (int)threadIdx.x < n) {
      double u[3];
      vertex_u(idx2, vt, jb + threadIdx.x, u);
      for (int k = 0; k < 3; ++k) { su[k][threadIdx.x] = u[k]; sq[k][threadIdx.x] = idx2[3 * (jb + threadIdx.x) + k]; }
    }
    __syncthreads();
    if (i >= n) continue;
    const int jend = min(kNaTile, n - jb);
    for (int jj = 0; jj < jend; ++jj) {
      const int j = jb + jj;
      if (j <= i) continue;
      const double d2 = pin_d2(ui[0], ui[1], ui[2], su[0][jj], su[1][jj], su[2][jj], sx, sy, sz);
      na_take(b[0], d2, i, j);
      const bool same_z = vt ? ui[2] == su[2][jj] : qi[2] == sq[2][jj];
      const bool same_y = vt ? ui[1] == su[1][jj] : qi[1] == sq[1][jj];
      const bool same_x = vt ? ui[0] == su[0][jj] : qi[0] == sq[0][jj];
      if (same_z) na_take(b[1], d2, i, j);
      if (same_y) na_take(b[2], d2, i, j);
      if (same_x) na_take(b[3], d2, i, j);
    }
  }
}

__global__ void __launch_bounds__(kNaTile) k_na_rows(const int16_t* idx2, const double* vt,
                                                     int n, double sx, double sy, double sz,
                                                     NaBest* slots) {
  pdl_enter();
  __shared__ double su[3][kNaTile];
  __shared__ int sq[3][kNaTile];
  __shared__ NaBest sred[4][kNaTile / 32];
  const int nt = (n + kNaTile - 1) / kNaTile;
  const int c = blockIdx.x;
  NaBest b[4];
  for (int q = 0; q < 4; ++q) { b[q].d2 = 0.0; b[q].i = -1; b[q].j = -1; }
  na_row(idx2, vt, n, nt, c, sx, sy, sz, su, sq, b);
  if (nt - 1 - c > c) na_row(idx2, vt, n, nt, nt - 1 - c, sx, sy, sz, su, sq, b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      NaBest o;
      o.d2 = __shfl_xor_sync(0xffffffffu, b[q].d2, off);
      o.i = __shfl_xor_sync(0xffffffffu, b[q].i, off);
      o.j = __shfl_xor_sync(0xffffffffu, b[q].j, off);
      if (na_better(o.d2, o.i, o.j, b[q])) b[q] = o;
    }
    if (lane == 0) sred[q][wid] = b[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    NaBest r = sred[q][0];
    for (int w = 1; w < kNaTile / 32; ++w)
      if (na_better(sred[q][w].d2, sred[q][w].i, sred[q][w].j, r)) r = sred[q][w];
    slots[4 * c + q] = r;
  }
}

__global__ void k_na_final(const NaBest* slots, int tiles, double* d2_out,
                           int32_t* pairs_out) {
  pdl_enter();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    NaBest r;
    r.d2 = 0.0; r.i = -1; r.j = -1;
    for (int t = 0; t < tiles; ++t)
      if (na_better(slots[4 * t + q].d2, slots[4 * t + q].i, slots[4 * t + q].j, r)) r = slots[4 * t + q];
    d2_out[q] = r.i >= 0 ? r.d2 : 0.0;
    pairs_out[2 * q] = r.i;
    pairs_out[2 * q + 1] = r.j;
  }
}

// Device address of the static scratch, looked up once per device (with that
// device current) and cached for the life of the process: a device reset
// (cudaDeviceReset) or any teardown of the device's primary context
// invalidates it, so the library must not be used across one.
std::mutex g_na_mu;
NaBest* g_na_ptr[64] = {nullptr};

rad_status na_scratch(NaBest** out) {
  int dev = 0;
  RAD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range for the static scratch table", dev);
    return RAD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    RAD_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_ptr[dev] = static_cast<NaBest*>(p);
  }
  *out = g_na_ptr[dev];
  return RAD_OK;
}

}  // namespace
}  // namespace rad

using namespace rad;

extern "C" rad_status rad_diameters_plain_fp64_noalloc(const int16_t* idx2_dev, const double* t_dev,
                                                       int64_t n_vertices, const double spacing[3], double* d2_dev,
                                                       int32_t* pairs_dev, void* stream) {
  if (!idx2_dev || !spacing || !d2_dev || !pairs_dev) {
    set_error("idx2_dev, spacing, d2_dev and pairs_dev must be non-NULL");
    return RAD_ERR_INVALID_ARG;
  }
  for (int k = 0; k < 3; ++k)
    if (!(spacing[k] > 0.0) || !isfinite(spacing[k])) {
      set_error("spacing[%d] = %g must be finite and > 0", k, spacing[k]);
      return RAD_ERR_INVALID_ARG;
    }
  const long long max_vertices = (long long)kNaMaxTiles * kNaTile;
  if (n_vertices < 0 || n_vertices > max_vertices) {
    set_error("n_vertices = %lld: the static scratch of this entry point holds %d tiles of %d vertices "
              "(at most %lld vertices)", (long long)n_vertices, kNaMaxTiles, kNaTile, max_vertices);
    return RAD_ERR_INVALID_ARG;
  }
  NaBest* slots = nullptr;
  RAD_TRY(na_scratch(&slots));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)n_vertices;
  const int tiles = (n + kNaTile - 1) / kNaTile;
  const int ctas = (tiles + 1) / 2;  // rows c and tiles - 1 - c per CTA
  if (ctas > 0)
    RAD_LAUNCH("noalloc_plain_fp64_rows", k_na_rows, ctas, kNaTile, 0, st, idx2_dev, t_dev, n, spacing[0], spacing[1],
               spacing[2], slots);
  RAD_LAUNCH("noalloc_plain_fp64_final", k_na_final, 1, 32, 0, st, slots, ctas, d2_dev, pairs_dev);
  return RAD_OK;
}
