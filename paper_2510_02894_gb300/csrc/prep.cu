// Preprocessing on the GPU: crop a mask to the bounding box of its region of
// interest and resample it by nearest neighbour (the step the paper leaves
// open, Sec. 3, "Discussion of the results": reading, cleaning and re-laying
// out the data before the features).  The definitions (ROI voxels, box,
// padding, output size, index maps, all in FP64 left to right):
//   ROI voxel   value == label (label >= 0) or value != 0 (label < 0)
//   box         per axis the smallest and largest ROI index, widened by pad
//               and clamped to the grid: lo_k .. hi_k, m_k = hi_k - lo_k + 1
//   resample    n'_k = floor((m_k - 1) s_k / s'_k) + 1 output voxels; output
//               voxel i samples lo_k + min(m_k - 1, floor(i s'_k / s_k + 1/2))
//   output      1 where the sampled voxel is an ROI voxel, else 0
//
// Three kernels: a bounding-box reduction over the mask (16 bytes per load
// where rows allow it, four bytes tested per instruction; its last block
// derives the box and the output size), the three per-axis index maps, and a
// gather that writes sixteen output voxels per thread.
#include <limits.h>

#include "rad_internal.cuh"

namespace rad {
namespace {

__device__ __forceinline__ bool roi_byte(unsigned int b, int label) {
  return label < 0 ? b != 0u : b == (unsigned int)label;
}

// The four bytes of v that are ROI voxels as 4 bits (byte k -> bit k), all
// four tested at once: a non-zero test (label < 0), or a zero test of v XOR
// the label replicated into every byte.
__device__ __forceinline__ uint32_t roi4(uint32_t v, int label) {
  const uint32_t x = label < 0 ? v : v ^ (0x01010101u * (uint32_t)label);
  uint32_t t = (x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;  // bit 7 of a byte set iff the byte of x is non-zero
  t = (t | x) & 0x80808080u;
  if (label >= 0) t ^= 0x80808080u;               // equal to the label: x's byte is zero
  return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// Lowest and highest set bit positions of a 16-bit mask (mask != 0).
__device__ __forceinline__ void bit_range(unsigned int m, int& lo, int& hi) {
  lo = __ffs(m) - 1;
  hi = 31 - __clz(m);
}

constexpr int kPrepThreads = 256;

__global__ void __launch_bounds__(kPrepThreads) k_prep_bbox(const uint8_t* mask, int nx, int ny, int nz, int label,
                                                            int vec16, int pad, double sx, double sy, double sz,
                                                            double tx, double ty, double tz, int resample, int* box,
                                                            PrepInfo* info, unsigned int* ticket) {
  pdl_enter();
  // 16-voxel chunks; the host keeps their count below 2^31, so the index
  // arithmetic is 32-bit
  const unsigned int cpr = vec16 ? nx / 16 : (nx + 15) / 16;
  const unsigned int total = cpr * (unsigned int)ny * (unsigned int)nz;
  int bmin[3] = {INT_MAX, INT_MAX, INT_MAX}, bmax[3] = {-1, -1, -1};
  for (unsigned int c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
    const unsigned int row = c / cpr;
    const int x0 = (int)(c - row * cpr) * 16;
    const uint8_t* p = mask + (long long)row * nx + x0;
    unsigned int m = 0u;
    if (vec16) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
      m = roi4(v.x, label) | (roi4(v.y, label) << 4) | (roi4(v.z, label) << 8) | (roi4(v.w, label) << 12);
    } else {
      const int nb = min(16, nx - x0);
      for (int k = 0; k < nb; ++k) m |= (unsigned int)roi_byte(__ldg(p + k), label) << k;
    }
    if (m == 0u) continue;
    int lo, hi;
    bit_range(m, lo, hi);
    const unsigned int z = row / (unsigned int)ny;
    const int y = (int)(row - z * (unsigned int)ny);
    bmin[0] = min(bmin[0], x0 + lo);
    bmax[0] = max(bmax[0], x0 + hi);
    bmin[1] = min(bmin[1], y);
    bmax[1] = max(bmax[1], y);
    bmin[2] = min(bmin[2], (int)z);
    bmax[2] = max(bmax[2], (int)z);
  }
  // warp, then block, then one atomic per value and block
  __shared__ int s_min[3][kPrepThreads / 32], s_max[3][kPrepThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = __reduce_min_sync(0xffffffffu, bmin[k]);
    const int b = __reduce_max_sync(0xffffffffu, bmax[k]);
    if (lane == 0) { s_min[k][wid] = a; s_max[k][wid] = b; }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int a = INT_MAX, b = -1;
    for (int w = 0; w < kPrepThreads / 32; ++w) {
      a = min(a, s_min[threadIdx.x][w]);
      b = max(b, s_max[threadIdx.x][w]);
    }
    if (b >= 0) {
      atomicMin(&box[threadIdx.x], a);
      atomicMax(&box[3 + threadIdx.x], b);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  PrepInfo r;
  const int n[3] = {nx, ny, nz};
  const double s[3] = {sx, sy, sz}, t[3] = {tx, ty, tz};
  r.empty = __ldcg(&box[3]) < 0;
  for (int k = 0; k < 3; ++k) {
    if (r.empty) {
      r.lo[k] = r.m[k] = r.nout[k] = 0;
      continue;
    }
    r.lo[k] = max(0, __ldcg(&box[k]) - pad);
    const long long hi = min((long long)n[k] - 1, (long long)__ldcg(&box[3 + k]) + pad);
    r.m[k] = hi - r.lo[k] + 1;
    r.nout[k] = resample ? (long long)floor(__ddiv_rn(__dmul_rn((double)(r.m[k] - 1), s[k]), t[k])) + 1 : r.m[k];
  }
  *info = r;
  *ticket = 0u;
}

// Input index (in the grid) of every output voxel, per axis: x, then y, then z.
__global__ void k_prep_maps(const PrepInfo* info, double sx, double sy, double sz, double tx, double ty, double tz,
                            int resample, int* maps) {
  pdl_enter();
  const PrepInfo r = *info;
  const long long total = r.nout[0] + r.nout[1] + r.nout[2];
  const double s[3] = {sx, sy, sz}, t[3] = {tx, ty, tz};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = e < r.nout[0] ? 0 : (e < r.nout[0] + r.nout[1] ? 1 : 2);
    const long long i = e - (k > 0 ? r.nout[0] : 0) - (k > 1 ? r.nout[1] : 0);
    long long off = i;
    if (resample) {
      const double x = __dadd_rn(__ddiv_rn(__dmul_rn((double)i, t[k]), s[k]), 0.5);
      off = min((long long)floor(x), r.m[k] - 1);
    }
    maps[e] = (int)(r.lo[k] + off);
  }
}

// Output voxels, sixteen consecutive bytes of the flat output per thread,
// whatever the row length: the first byte's (x, y, z) from one division, then
// x stepped (and the row advanced at its end); one 16-byte store when the
// output is 16-byte aligned and the run is whole.
__global__ void __launch_bounds__(kPrepThreads) k_prep_gather(const uint8_t* mask, int nx, int ny, int label,
                                                              const PrepInfo* info, const int* maps, uint8_t* out) {
  pdl_enter();
  const PrepInfo r = *info;
  const long long ox = r.nout[0], oy = r.nout[1], oz = r.nout[2];
  const long long total = ox * oy * oz;  // with the runs below 2^31 x 16 (checked on the host)
  const unsigned int runs = (unsigned int)((total + 15) / 16);
  const int* mx = maps;
  const int* my = maps + ox;
  const int* mz = my + oy;
  const bool aligned = ((uintptr_t)out & 15) == 0;
  const unsigned int ox32 = (unsigned int)ox, oy32 = (unsigned int)oy;
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < runs; e += gridDim.x * blockDim.x) {
    const long long f0 = (long long)e * 16;
    unsigned int row = (unsigned int)(f0 / ox32);
    unsigned int x = (unsigned int)(f0 - (long long)row * ox32);
    unsigned int z = row / oy32, y = row - z * oy32;
    const uint8_t* src = mask + ((long long)__ldg(&mz[z]) * ny + __ldg(&my[y])) * nx;
    const int nb = (int)min(16ll, total - f0);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (int k = 0; k < nb; ++k) {
      w[k >> 2] |= (uint32_t)roi_byte(__ldg(src + __ldg(&mx[x])), label) << (8 * (k & 3));
      if (++x == ox32 && k + 1 < nb) {  // next output row
        x = 0;
        if (++y == oy32) { y = 0; ++z; }
        src = mask + ((long long)__ldg(&mz[z]) * ny + __ldg(&my[y])) * nx;
      }
    }
    uint8_t* dst = out + f0;
    if (aligned && nb == 16) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      for (int k = 0; k < nb; ++k) dst[k] = (uint8_t)((w[k >> 2] >> (8 * (k & 3))) & 0xffu);
    }
  }
}

}  // namespace

rad_status prep_bbox(const uint8_t* mask, const int64_t dims[3], const double sp[3], int label, int pad,
                     const double* new_sp, DevBuf& scratch, PrepInfo* info_host, cudaStream_t st) {
  const int nx = (int)dims[0], ny = (int)dims[1], nz = (int)dims[2];
  RAD_TRY(scratch.reserve(256));
  char* base = scratch.as<char>();
  int* box = reinterpret_cast<int*>(base);                       // 6 ints
  unsigned int* ticket = reinterpret_cast<unsigned int*>(base + 32);
  PrepInfo* info = reinterpret_cast<PrepInfo*>(base + 64);
  RAD_CUDA(cudaMemsetAsync(box, 0x7f, sizeof(int) * 3, st));       // minima: 0x7f7f7f7f
  RAD_CUDA(cudaMemsetAsync(box + 3, 0xff, sizeof(int) * 3, st));   // maxima: -1
  RAD_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
  const int vec16 = (nx % 16) == 0 && (((uintptr_t)mask) & 15) == 0;
  const long long chunks = (long long)(vec16 ? nx / 16 : (nx + 15) / 16) * ny * nz;
  const double t[3] = {new_sp ? new_sp[0] : sp[0], new_sp ? new_sp[1] : sp[1], new_sp ? new_sp[2] : sp[2]};
  RAD_LAUNCH("prep_bbox", k_prep_bbox, wave_grid(k_prep_bbox, kPrepThreads, (chunks + kPrepThreads - 1) / kPrepThreads),
             kPrepThreads, 0, st, mask, nx, ny, nz, label, vec16, pad, sp[0], sp[1], sp[2], t[0], t[1], t[2],
             new_sp ? 1 : 0, box, info, ticket);
  RAD_CUDA(cudaMemcpyAsync(info_host, info, sizeof(PrepInfo), cudaMemcpyDeviceToHost, st));
  RAD_CUDA(cudaStreamSynchronize(st));
  return RAD_OK;
}

rad_status prep_gather(const uint8_t* mask, const int64_t dims[3], const double sp[3], int label,
                       const double* new_sp, const PrepInfo& info_host, DevBuf& scratch, uint8_t* out,
                       cudaStream_t st) {
  const long long nmap = info_host.nout[0] + info_host.nout[1] + info_host.nout[2];
  // the box result stays where prep_bbox put it (offset 64); the maps follow
  PrepInfo saved = info_host;
  DevBuf& sb = scratch;
  if (sb.bytes < 256 + sizeof(int) * (size_t)nmap) {
    // growing the buffer moves it: carry the device copy of the box result along
    RAD_TRY(sb.reserve(256 + sizeof(int) * (size_t)nmap));
    RAD_CUDA(cudaMemcpyAsync(sb.as<char>() + 64, &saved, sizeof(PrepInfo), cudaMemcpyHostToDevice, st));
  }
  const PrepInfo* info = reinterpret_cast<const PrepInfo*>(sb.as<char>() + 64);
  int* maps = reinterpret_cast<int*>(sb.as<char>() + 256);
  const double t[3] = {new_sp ? new_sp[0] : sp[0], new_sp ? new_sp[1] : sp[1], new_sp ? new_sp[2] : sp[2]};
  RAD_LAUNCH("prep_maps", k_prep_maps, wave_grid(k_prep_maps, 256, (nmap + 255) / 256), 256, 0, st, info, sp[0],
             sp[1], sp[2], t[0], t[1], t[2], new_sp ? 1 : 0, maps);
  const long long runs = (info_host.nout[0] * info_host.nout[1] * info_host.nout[2] + 15) / 16;
  RAD_LAUNCH("prep_gather", k_prep_gather,
             wave_grid(k_prep_gather, kPrepThreads, (runs + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0, st,
             mask, (int)dims[0], (int)dims[1], label, info, maps, out);
  RAD_CUDA(cudaStreamSynchronize(st));  // a host copy of the box result may have been the source above
  return RAD_OK;
}

}  // namespace rad
