// Adjoint of the soft-map shape features: gradient of
//   L = gA * SurfaceArea + gV * MeshVolume + sum_q gD_q * D_q
// (D_q: the maximum 3D, Slice, Column and Row diameters) with respect to
// every voxel value of each float32 probability map of a batch, whose
// iso-0.5 mesh has linearly interpolated vertices (the soft extension of the
// marching cubes of Sec. 2; the paper itself has no gradient).
//
// The mesh is recomputed (not stored) before these kernels run.  Topology,
// triangulation choice and the argmax pair of the diameter are held fixed
// (piecewise-differentiable reading):
//   per triangle (a, b, c), n = (b - a) x (c - a), n^ = n / |n|:
//     dA/da = (b - c) x n^ / 2,  dA/db = (c - a) x n^ / 2,  dA/dc = (a - b) x n^ / 2
//     dV/da = (b x c) / 6,       dV/db = (c x a) / 6,       dV/dc = (a x b) / 6
//   argmax pair (i, j) of each diameter, D = |p_i - p_j|:
//     dD/dp_i = (p_i - p_j) / D = -dD/dp_j   (a planar pair's plane held fixed)
//   vertex on the edge (g, g + e_axis), t = (1/2 - v0) / (v1 - v0):
//     dp_axis/dt = s_axis,  dt/dv0 = (1/2 - v1) / (v1 - v0)^2,
//     dt/dv1 = -(1/2 - v0) / (v1 - v0)^2
// Vertex and voxel sums use FP64 atomics (rounding-order differences only).
#include <algorithm>

#include "rad_internal.cuh"

namespace rad {
namespace {

// O-relative physical position of vertex v (O = centre of the padded box).
__device__ __forceinline__ void soft_pos(const int16_t* idx2, const double* vt, long long v, const MeshDims& d,
                                         const double* sp, double P[3]) {
  const int n[3] = {d.nx, d.ny, d.nz};
  const double t = vt[v];
  for (int k = 0; k < 3; ++k) {
    const int q = idx2[3 * v + k];
    const int g = (q - (q & 1)) >> 1;  // owner index (floor of q / 2)
    P[k] = ((double)g - 0.5 * (double)(n[k] - 1) + ((q & 1) ? t : 0.0)) * sp[k];
  }
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Map of a global vertex or triangle id: last ROI whose first id is <= v.
__device__ __forceinline__ int roi_of(const RoiOut* ro, int n, long long v, bool tris) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((tris ? ro[mid].t0 : ro[mid].v0) <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ MeshDims dims_of(const SoftMap& m) { return MeshDims{m.nx, m.ny, m.nz}; }

__global__ void k_soft_tri_grad(const int16_t* idx2, const double* vt, const int32_t* tri, const long long* nt_dev,
                                long long tcap, const RoiOut* ro, const SoftMap* maps, int n, double* gvtx) {
  pdl_enter();
  const long long nt = min(*nt_dev, tcap);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
    const SoftMap& m = maps[n == 1 ? 0 : roi_of(ro, n, t, true)];
    const double gA = m.gout[0], gV = m.gout[1];
    if (gA == 0.0 && gV == 0.0) continue;
    const MeshDims d = dims_of(m);
    const double sp[3] = {m.sx, m.sy, m.sz};
    const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
    double a[3], b[3], c[3];
    soft_pos(idx2, vt, ia, d, sp, a);
    soft_pos(idx2, vt, ib, d, sp, b);
    soft_pos(idx2, vt, ic, d, sp, c);
    double ga[3] = {0, 0, 0}, gb[3] = {0, 0, 0}, gc[3] = {0, 0, 0};
    if (gA != 0.0) {
      double e1[3], e2[3], nrm[3];
      for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
      cross3(e1, e2, nrm);
      const double nn = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
      if (nn > 0.0) {
        const double nh[3] = {nrm[0] / nn, nrm[1] / nn, nrm[2] / nn};
        double bc[3], ca[3], ab[3], x[3];
        for (int k = 0; k < 3; ++k) { bc[k] = b[k] - c[k]; ca[k] = c[k] - a[k]; ab[k] = a[k] - b[k]; }
        cross3(bc, nh, x);
        for (int k = 0; k < 3; ++k) ga[k] += gA * 0.5 * x[k];
        cross3(ca, nh, x);
        for (int k = 0; k < 3; ++k) gb[k] += gA * 0.5 * x[k];
        cross3(ab, nh, x);
        for (int k = 0; k < 3; ++k) gc[k] += gA * 0.5 * x[k];
      }
    }
    if (gV != 0.0) {
      double x[3];
      cross3(b, c, x);
      for (int k = 0; k < 3; ++k) ga[k] += gV * x[k] / 6.0;
      cross3(c, a, x);
      for (int k = 0; k < 3; ++k) gb[k] += gV * x[k] / 6.0;
      cross3(a, b, x);
      for (int k = 0; k < 3; ++k) gc[k] += gV * x[k] / 6.0;
    }
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&gvtx[3 * (long long)ia + k], ga[k]);
      atomicAdd(&gvtx[3 * (long long)ib + k], gb[k]);
      atomicAdd(&gvtx[3 * (long long)ic + k], gc[k]);
    }
  }
}

// One thread per (map, diameter): the argmax pair's two position gradients.
// A pair that is not a vertex pair of its map's mesh (one side negative, out
// of range or both equal) raises DEV_ERR_PAIR and adds nothing.
__global__ void k_soft_pair_grad(const int16_t* idx2, const double* vt, const RoiOut* ro, const SoftMap* maps, int n,
                                 double* gvtx, unsigned int* status) {
  pdl_enter();
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= 4 * n) return;
  const SoftMap& m = maps[it >> 2];
  const int q = it & 3;
  const double gD = m.gout[2 + q];
  const int il = m.pair[2 * q], jl = m.pair[2 * q + 1];
  if (il < 0 && jl < 0) return;
  const long long nv = ro[it >> 2].nv;
  if (il < 0 || jl < 0 || il >= nv || jl >= nv || il == jl) {
    atomicOr(status, DEV_ERR_PAIR);
    return;
  }
  if (gD == 0.0) return;
  const long long v0 = ro[it >> 2].v0, i = v0 + il, j = v0 + jl;
  const MeshDims d = dims_of(m);
  const double sp[3] = {m.sx, m.sy, m.sz};
  double pi[3], pj[3], df[3];
  soft_pos(idx2, vt, i, d, sp, pi);
  soft_pos(idx2, vt, j, d, sp, pj);
  for (int k = 0; k < 3; ++k) df[k] = pi[k] - pj[k];
  const double D = sqrt(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
  if (!(D > 0.0)) return;
  for (int k = 0; k < 3; ++k) {
    atomicAdd(&gvtx[3 * i + k], gD * df[k] / D);
    atomicAdd(&gvtx[3 * j + k], -gD * df[k] / D);
  }
}

__device__ __forceinline__ double voxel(const float* p, const MeshDims& d, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0.0;
  return (double)__ldg(p + ((long long)z * d.ny + y) * d.nx + x);
}

// Every map's gradient to zero (one grid over all maps' voxels).
__global__ void k_soft_zero(const SoftMap* maps, int n, long long total) {
  pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (maps[mid].vox0 <= e) lo = mid;
      else hi = mid - 1;
    }
    maps[lo].grad[e - maps[lo].vox0] = 0.0;
  }
}

__global__ void k_soft_scatter(const int16_t* idx2, const long long* nv_dev, long long vcap, const RoiOut* ro,
                               const SoftMap* maps, int n, const double* gvtx) {
  pdl_enter();
  const long long nv = min(*nv_dev, vcap);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    const SoftMap& m = maps[n == 1 ? 0 : roi_of(ro, n, v, false)];
    const MeshDims d = dims_of(m);
    const double sp[3] = {m.sx, m.sy, m.sz};
    int g[3], a = 0;
    for (int k = 0; k < 3; ++k) {
      const int q = idx2[3 * v + k];
      g[k] = (q - (q & 1)) >> 1;
      if (q & 1) a = k;
    }
    const double dLdt = gvtx[3 * v + a] * sp[a];
    if (dLdt == 0.0) continue;
    const double v0 = voxel(m.prob, d, g[0], g[1], g[2]);
    const double v1 = voxel(m.prob, d, g[0] + (a == 0), g[1] + (a == 1), g[2] + (a == 2));
    const double den = (v1 - v0) * (v1 - v0);
    const double d0 = (0.5 - v1) / den, d1 = -(0.5 - v0) / den;
    if (g[0] >= 0 && g[1] >= 0 && g[2] >= 0 && g[0] < d.nx && g[1] < d.ny && g[2] < d.nz)
      atomicAdd(&m.grad[((long long)g[2] * d.ny + g[1]) * d.nx + g[0]], dLdt * d0);
    const int h[3] = {g[0] + (a == 0), g[1] + (a == 1), g[2] + (a == 2)};
    if (h[0] < d.nx && h[1] < d.ny && h[2] < d.nz && h[0] >= 0 && h[1] >= 0 && h[2] >= 0)
      atomicAdd(&m.grad[((long long)h[2] * d.ny + h[1]) * d.nx + h[0]], dLdt * d1);
  }
}

}  // namespace

rad_status soft_adjoint(const int16_t* idx2, const double* vt, const int32_t* tri, const long long* nv_dev,
                        const long long* nt_dev, long long vcap, long long tcap, const RoiOut* ro, const SoftMap* maps,
                        int n, long long total_vox, double* gvtx, unsigned int* status, cudaStream_t st) {
  const int sms = num_sms();
  RAD_CUDA(cudaMemsetAsync(gvtx, 0, sizeof(double) * 3 * std::max<long long>(vcap, 1), st));
  RAD_LAUNCH("soft_zero", k_soft_zero, wave_grid(k_soft_zero, 256, (total_vox + 255) / 256), 256, 0, st, maps, n,
             total_vox);
  RAD_LAUNCH("soft_tri_grad", k_soft_tri_grad, sms * 8, 256, 0, st, idx2, vt, tri, nt_dev, tcap, ro, maps, n, gvtx);
  RAD_LAUNCH("soft_pair_grad", k_soft_pair_grad, (4 * n + 127) / 128, 128, 0, st, idx2, vt, ro, maps, n, gvtx,
             status);
  RAD_LAUNCH("soft_scatter", k_soft_scatter, sms * 8, 256, 0, st, idx2, nv_dev, vcap, ro, maps, n, gvtx);
  return RAD_OK;
}

}  // namespace rad
