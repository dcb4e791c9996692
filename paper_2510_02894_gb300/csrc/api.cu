// C ABI of the shape-feature library (declared in include/rad.h): argument
// validation, library-owned device buffers, the launch sequence of each entry
// point, status words, per-kernel timing and error text.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "rad_internal.cuh"

namespace rad {

// ---- error text -----------------------------------------------------------------

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

rad_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? RAD_ERR_OOM : RAD_ERR_CUDA;
}

// ---- launch bookkeeping ------------------------------------------------------------

namespace {
struct Pending {
  int stat;
  cudaEvent_t a, b;
};
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<rad_kernel_stat_t> stats;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long long launches = 0;
};
Prof& prof() {
  static Prof* p = new Prof();
  return *p;
}
cudaEvent_t get_event(Prof& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
void flush_pending(Prof& p) {
  for (auto& q : p.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess)
      p.stats[q.stat].total_ms += ms;
    else
      cudaGetLastError();  // a timing failure must not surface in the caller's next CUDA call
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pending.clear();
}
}  // namespace

// While a CUDA graph is being captured on this thread, launches are collected
// here: their kernel-stat slots (counted per replay) and, with profiling on,
// the event pair around each kernel (recorded by every replay).
struct CaptureSink {
  std::vector<int> stats;
  std::vector<Pending> slots;
};
static thread_local CaptureSink* g_sink = nullptr;

void launch_begin(const char* name, cudaStream_t s, void** token) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.launches++;
  int idx = -1;
  for (size_t i = 0; i < p.stats.size(); ++i)
    if (strncmp(p.stats[i].name, name, sizeof(p.stats[i].name)) == 0) { idx = (int)i; break; }
  if (idx < 0) {
    rad_kernel_stat_t st;
    memset(&st, 0, sizeof(st));
    strncpy(st.name, name, sizeof(st.name) - 1);
    p.stats.push_back(st);
    idx = (int)p.stats.size() - 1;
  }
  p.stats[idx].launches++;
  if (g_sink) g_sink->stats.push_back(idx);
  if (!p.on) {
    *token = nullptr;
    return;
  }
  Pending q;
  q.stat = idx;
  q.a = get_event(p);
  q.b = get_event(p);
  if (g_sink) {
    // inside a capture only an external record becomes a node that records
    // the event at every replay
    cudaEventRecordWithFlags(q.a, s, cudaEventRecordExternal);
    g_sink->slots.push_back(q);
    *token = reinterpret_cast<void*>((intptr_t)(-(intptr_t)g_sink->slots.size()));
    return;
  }
  cudaEventRecord(q.a, s);
  if (p.pending.size() > 4096) flush_pending(p);
  p.pending.push_back(q);
  *token = reinterpret_cast<void*>((intptr_t)p.pending.size());
}

bool profiling_on() {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  return p.on;
}

void launch_end(void* token, cudaStream_t s) {
  if (!token) return;
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  const intptr_t t = (intptr_t)token;
  if (t < 0) {
    if (g_sink && (size_t)(-t - 1) < g_sink->slots.size())
      cudaEventRecordWithFlags(g_sink->slots[-t - 1].b, s, cudaEventRecordExternal);
    return;
  }
  const size_t i = (size_t)t - 1;
  if (i < p.pending.size()) cudaEventRecord(p.pending[i].b, s);
}

// Bookkeeping of a captured graph: undo the counts made while capturing, then
// add one launch per captured kernel at every replay and, after the replay has
// finished, the elapsed time of each captured event pair.
void graph_undo_capture(const CaptureSink& k) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.launches -= (long long)k.stats.size();
  for (int i : k.stats) p.stats[i].launches--;
}

void graph_replayed(const CaptureSink& k) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.launches += (long long)k.stats.size();
  for (int i : k.stats) p.stats[i].launches++;
}

void graph_timed(const CaptureSink& k) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  for (const Pending& q : k.slots) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) p.stats[q.stat].total_ms += ms;
    else cudaGetLastError();
  }
}

void graph_release(CaptureSink& k) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  for (const Pending& q : k.slots) {
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  k.slots.clear();
  k.stats.clear();
}

int resident_ctas(const void* kernel, int threads, size_t smem) {
  struct Key {
    const void* k;
    int threads, dev;
    size_t smem;
    int n;
  };
  static std::mutex mu;
  static std::vector<Key> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  for (const Key& e : cache)
    if (e.k == kernel && e.threads == threads && e.dev == dev && e.smem == smem) return e.n;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  n = std::max(n, 1);
  cache.push_back(Key{kernel, threads, dev, smem, n});
  return n;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 132;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 132;
  }
  return cached[dev];
}

// ---- buffers -----------------------------------------------------------------------

static std::atomic<long long> g_alloc_epoch{0};
long long alloc_epoch() { return g_alloc_epoch.load(); }

rad_status DevBuf::reserve(size_t need) {
  if (need <= bytes && p) return RAD_OK;
  g_alloc_epoch++;
  if (p) {
    cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  size_t n = std::max<size_t>(need + need / 4, 256);
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed: %s", n, cudaGetErrorString(e));
    return RAD_ERR_OOM;
  }
  bytes = n;
  return RAD_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

static rad_tuning_t g_tuning = {128, 128, 8, 4};
const rad_tuning_t& tuning() { return g_tuning; }

// ---- per-workspace state --------------------------------------------------------------

struct ResultBlock {  // device; copied to pinned host memory after every pass (8-byte aligned POD)
  MeshTotals tot;
  DiamStats stats;
};

// One warp looks back from chunk 1 at chunk 0, which never publishes: the
// bounded wait gives up and raises DEV_ERR_TIMEOUT.
__global__ void k_wait_probe(ScanTile<1>* tiles, unsigned int* status) {
  pdl_enter();
  long long e = 0;
  scan_lookback(tiles, 1, &e, status);
}

// Features of every ROI from the mesh and diameter results (one thread per
// ROI), written straight into the caller-visible pinned host buffer (mapped
// into the device's address space), and the pass's result block copied to
// its pinned host copy by the first threads: no copy nodes after the pass.
__global__ void k_assemble(const Roi* rois, const RoiOut* ro,
                           const DiamOut* dout, int n, int have_diam, rad_features_t* f,
                           const ResultBlock* res, ResultBlock* res_host) {
  pdl_enter();
  static_assert(sizeof(ResultBlock) % 8 == 0, "result block copied in 8-byte words");
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < (int)(sizeof(ResultBlock) / 8); k += blockDim.x)
      reinterpret_cast<unsigned long long*>(res_host)[k] = reinterpret_cast<const unsigned long long*>(res)[k];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const Roi& r = rois[i];
    const RoiOut& o = ro[i];
    rad_features_t x;
    x.MeshVolume = o.vol6 / 6.0;
    x.SurfaceArea = o.area2 * 0.5;
    x.VoxelVolume = (double)o.nvox * r.sx * r.sy * r.sz;
    x.n_vertices = o.nv;
    x.n_triangles = o.nt;
    x.n_voxels = o.nvox;
    double* D[4] = {&x.Maximum3DDiameter, &x.Maximum2DDiameterSlice, &x.Maximum2DDiameterColumn,
                    &x.Maximum2DDiameterRow};
    int32_t* A[4] = {x.argmax3d, x.argmax_slice, x.argmax_column, x.argmax_row};
    for (int q = 0; q < 4; ++q) {
      const unsigned long long pr = have_diam ? dout[i].pair[q] : ~0ull;
      const bool ok = pr != ~0ull;
      *D[q] = ok ? sqrt(__longlong_as_double((long long)dout[i].d2[q])) : 0.0;
      A[q][0] = ok ? (int32_t)(pr >> 32) : -1;
      A[q][1] = ok ? (int32_t)(pr & 0xffffffffu) : -1;
    }
    x.status = 0;
    x._pad = 0;
    double* dv[10] = {&x.Sphericity, &x.SurfaceVolumeRatio, &x.Compactness1, &x.Compactness2,
                      &x.SphericalDisproportion, &x.MajorAxisLength, &x.MinorAxisLength, &x.LeastAxisLength,
                      &x.Elongation, &x.Flatness};
    for (int k = 0; k < 10; ++k) *dv[k] = o.has_derived ? o.derived[k] : 0.0;
    f[i] = x;
  }
}

struct Work {
  MeshScratch ms;
  DiamScratch ds;
  DevBuf result;            // ResultBlock
  DevBuf ro, dout;          // per ROI: RoiOut, DiamOut
  DevBuf rois_dev, rd_dev;  // per ROI: Roi, RoiDiam
  DevBuf idx2, vt, tri;
  long long vcap = 0, tcap = 0;
  ResultBlock* host = nullptr;       // pinned copies, written by the assembly kernel
  rad_features_t* hfeats = nullptr;
  int hfeats_cap = 0;
  DevBuf mask;  // device copy of a host mask (rad_extract_host)
  DevBuf gvtx;  // per-vertex position gradients (soft adjoint)
  DevBuf plain; // result of the plain FP64 kernel
  DevBuf soft_maps;  // SoftMap table of a soft adjoint batch
  std::vector<SoftMap> soft_maps_host;  // its host copy (the source of the upload)
  std::vector<Roi> prev_rois;           // map table of the previous soft forward call
  DevBuf prep;       // crop/resample: box reduction, its result and the index maps
  // plan of the current batch
  std::vector<Roi> rois, up_rois;     // planned / last uploaded
  std::vector<RoiDiam> rd, up_rd;
  std::vector<double> tab_sp;         // spacings of the uploaded case tables
  MeshBatch mb;
  long long nkeys = 0, nplanes = 0, ntab = 0;
  bool soft = false;
  // side branch of a pass: the diameter stage's initialisation runs beside
  // the mesh, the masks' per-ROI totals beside the diameters
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_init = nullptr, ev_tot = nullptr, ev_cnt = nullptr;
  // CUDA graph of the whole pass, valid for the ROI table it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long g_epoch = -1;
  bool g_prof = false;
  std::vector<Roi> g_rois;
  std::vector<RoiDiam> g_rd;
  rad_tuning_t g_tuning = {0, 0, 0, 0};
  CaptureSink g_sink_data;
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    graph_release(g_sink_data);
  }
  ~Work() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side) cudaStreamDestroy(side);
    for (cudaEvent_t e : {ev_fork, ev_init, ev_tot, ev_cnt})
      if (e) cudaEventDestroy(e);
    for (DevBuf* b : {&ms.bits, &ms.counts, &ms.wpre, &ms.tpre, &ms.wlist, &ms.prefix, &ms.chunk, &ms.cubes, &ms.hist, &ms.partial,
                      &ms.bintab, &ms.tabsp, &ds.misc, &ds.plain_part, &result, &ro, &dout, &rois_dev,
                      &rd_dev, &idx2, &vt, &tri, &mask, &gvtx, &plain, &soft_maps, &prep})
      b->release();
    if (host) cudaFreeHost(host);
    if (hfeats) cudaFreeHost(hfeats);
  }
  ResultBlock* dres() const { return result.as<ResultBlock>(); }
  RoiOut* dro() const { return ro.as<RoiOut>(); }
};

static bool same_bytes(const void* a, const void* b, size_t n) { return memcmp(a, b, n) == 0; }

// Plan a batch (ROI table, case tables, diameter parameters) and upload what
// changed.  All uploads happen here, outside any graph capture.
static rad_status prepare(Work& w, int n, const void* const* data, const int64_t* dims, const double* sp, bool soft,
                          cudaStream_t st) {
  if (!w.host) RAD_CUDA(cudaMallocHost(&w.host, sizeof(ResultBlock)));
  if (w.hfeats_cap < n) {
    if (w.hfeats) cudaFreeHost(w.hfeats);
    w.hfeats = nullptr;
    RAD_CUDA(cudaMallocHost(&w.hfeats, sizeof(rad_features_t) * n));
    w.hfeats_cap = n;
  }
  RAD_TRY(w.result.reserve(sizeof(ResultBlock)));
  RAD_TRY(w.ro.reserve(sizeof(RoiOut) * n));
  RAD_TRY(w.dout.reserve(sizeof(DiamOut) * n));
  // case tables: one per distinct spacing (binary masks)
  std::vector<int> tab(n, 0);
  std::vector<double> tsp;
  if (!soft) {
    for (int i = 0; i < n; ++i) {
      int k = 0;
      for (; k < (int)tsp.size() / 3; ++k)
        if (tsp[3 * k] == sp[3 * i] && tsp[3 * k + 1] == sp[3 * i + 1] && tsp[3 * k + 2] == sp[3 * i + 2]) break;
      if (k == (int)tsp.size() / 3) tsp.insert(tsp.end(), {sp[3 * i], sp[3 * i + 1], sp[3 * i + 2]});
      tab[i] = k;
    }
    if (tsp != w.tab_sp) {
      RAD_TRY(mesh_tables(tsp.data(), (int)tsp.size() / 3, w.ms, st));
      w.tab_sp = tsp;
    }
  }
  plan_batch(dims, data, tab.data(), sp, n, soft, w.rois, w.mb);
  plan_diam(w.rois, soft, w.rd, w.nkeys, w.ntab, w.nplanes);
  w.soft = soft;
  RAD_TRY(w.rois_dev.reserve(sizeof(Roi) * n));
  RAD_TRY(w.rd_dev.reserve(sizeof(RoiDiam) * n));
  if (w.up_rois.size() != w.rois.size() || !same_bytes(w.up_rois.data(), w.rois.data(), sizeof(Roi) * n) ||
      w.up_rd.size() != w.rd.size() || !same_bytes(w.up_rd.data(), w.rd.data(), sizeof(RoiDiam) * n) ||
      w.rois_dev.p != w.mb.rois) {
    RAD_CUDA(cudaMemcpyAsync(w.rois_dev.p, w.rois.data(), sizeof(Roi) * n, cudaMemcpyHostToDevice, st));
    RAD_CUDA(cudaMemcpyAsync(w.rd_dev.p, w.rd.data(), sizeof(RoiDiam) * n, cudaMemcpyHostToDevice, st));
    RAD_CUDA(cudaStreamSynchronize(st));  // the host vectors may change before the copy runs
    w.up_rois = w.rois;
    w.up_rd = w.rd;
  }
  w.mb.rois = w.rois_dev.as<Roi>();
  return RAD_OK;
}

// Counting pass + exact pool sizing (synchronises).
static rad_status size_pools(Work& w, cudaStream_t st) {
  ResultBlock* dr = w.dres();
  RAD_TRY(mesh_count(w.mb, w.ms, &dr->tot, w.dro(), st));
  RAD_CUDA(cudaMemcpyAsync(w.host, dr, sizeof(ResultBlock), cudaMemcpyDeviceToHost, st));
  RAD_CUDA(cudaStreamSynchronize(st));
  const long long nv = w.host->tot.nv, nt = w.host->tot.nt;
  if (nv >= (1LL << 31) || nt >= (1LL << 31)) {
    set_error("mesh too large: %lld vertices, %lld triangles", nv, nt);
    return RAD_ERR_CAPACITY;
  }
  RAD_TRY(w.idx2.reserve(sizeof(int16_t) * 3 * std::max<long long>(nv, 1)));
  if (w.soft) RAD_TRY(w.vt.reserve(sizeof(double) * std::max<long long>(nv, 1)));
  RAD_TRY(w.tri.reserve(sizeof(int32_t) * 3 * std::max<long long>(nt, 1)));
  w.vcap = (long long)(w.idx2.bytes / (3 * sizeof(int16_t)));
  w.tcap = (long long)(w.tri.bytes / (3 * sizeof(int32_t)));
  if (w.soft) w.vcap = std::min<long long>(w.vcap, (long long)(w.vt.bytes / sizeof(double)));
  return RAD_OK;
}

static rad_status enqueue_mesh(Work& w, cudaStream_t st, bool count) {
  ResultBlock* dr = w.dres();
  if (count) RAD_TRY(mesh_count(w.mb, w.ms, &dr->tot, w.dro(), st));
  RAD_TRY(mesh_moments(w.mb, w.ms, &dr->tot, w.dro(), st));
  return mesh_emit(w.mb, w.ms, &dr->tot, w.dro(), w.idx2.as<int16_t>(), w.soft ? w.vt.as<double>() : nullptr,
                   w.tri.as<int32_t>(), w.vcap, w.tcap, st);
}

static rad_status enqueue_shape(Work& w, cudaStream_t st) {
  ResultBlock* dr = w.dres();
  RAD_TRY(diam_run(w.mb.n, w.rd_dev.as<RoiDiam>(), w.dro(), &dr->tot.nv, w.vcap, w.nkeys, w.nplanes, w.ntab,
                   true, w.idx2.as<int16_t>(), w.soft ? w.vt.as<double>() : nullptr, w.ds, w.dout.as<DiamOut>(),
                   &dr->stats, st));
  return RAD_OK;
}

static rad_status enqueue_finish(Work& w, bool have_diam, cudaStream_t st) {
  const int n = w.mb.n;
  RAD_LAUNCH("assemble", k_assemble, std::max(1, (n + 127) / 128), 128, 0, st, w.mb.rois, w.dro(),
             w.dout.as<DiamOut>(), n, have_diam ? 1 : 0, w.hfeats, w.dres(), w.host);
  return RAD_OK;
}

// One whole pass (mesh, diameters, features to pinned host memory).  The
// diameter stage's initialisation depends on nothing from the mesh, and the
// voxel moments and the masks' per-ROI totals feed only the final assembly:
// they run on a side branch (two branches of one graph when captured).  With per-kernel
// profiling on, the pass stays on one stream so every kernel is timed alone.
static rad_status enqueue_pass(Work& w, cudaStream_t st) {
  if (profiling_on()) {
    RAD_TRY(enqueue_mesh(w, st, true));
    RAD_TRY(enqueue_shape(w, st));
    return enqueue_finish(w, true, st);
  }
  if (!w.side) RAD_CUDA(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&w.ev_fork, &w.ev_init, &w.ev_tot, &w.ev_cnt})
    if (!*e) RAD_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  ResultBlock* dr = w.dres();
  RAD_CUDA(cudaEventRecord(w.ev_fork, st));
  RAD_CUDA(cudaStreamWaitEvent(w.side, w.ev_fork, 0));
  RAD_TRY(diam_run(w.mb.n, w.rd_dev.as<RoiDiam>(), w.dro(), &dr->tot.nv, w.vcap, w.nkeys, w.nplanes, w.ntab,
                   true, w.idx2.as<int16_t>(), w.soft ? w.vt.as<double>() : nullptr, w.ds, w.dout.as<DiamOut>(),
                   &dr->stats, w.side, 1));
  RAD_CUDA(cudaEventRecord(w.ev_init, w.side));
  RAD_TRY(mesh_count(w.mb, w.ms, &dr->tot, w.dro(), st));
  // the voxel moments need only the packed bits: beside the emit pass
  RAD_CUDA(cudaEventRecord(w.ev_cnt, st));
  RAD_CUDA(cudaStreamWaitEvent(w.side, w.ev_cnt, 0));
  RAD_TRY(mesh_moments(w.mb, w.ms, &dr->tot, w.dro(), w.side));
  RAD_TRY(mesh_emit(w.mb, w.ms, &dr->tot, w.dro(), w.idx2.as<int16_t>(), w.soft ? w.vt.as<double>() : nullptr,
                    w.tri.as<int32_t>(), w.vcap, w.tcap, st, false));
  RAD_CUDA(cudaEventRecord(w.ev_fork, st));
  RAD_CUDA(cudaStreamWaitEvent(w.side, w.ev_fork, 0));
  RAD_TRY(mesh_totals(w.mb, w.ms, w.dro(), w.side));
  RAD_CUDA(cudaEventRecord(w.ev_tot, w.side));
  RAD_CUDA(cudaStreamWaitEvent(st, w.ev_init, 0));
  RAD_TRY(diam_run(w.mb.n, w.rd_dev.as<RoiDiam>(), w.dro(), &dr->tot.nv, w.vcap, w.nkeys, w.nplanes, w.ntab,
                   true, w.idx2.as<int16_t>(), w.soft ? w.vt.as<double>() : nullptr, w.ds, w.dout.as<DiamOut>(),
                   &dr->stats, st, 2));
  RAD_CUDA(cudaStreamWaitEvent(st, w.ev_tot, 0));
  return enqueue_finish(w, true, st);
}

// Capture the pass into a CUDA graph on an internal stream (the caller's
// stream may be the legacy default stream, which cannot be captured).  Every
// buffer is already sized by an eager pass, so nothing is allocated inside.
static rad_status capture_pass(Work& w) {
  w.drop_graph();
  if (!w.cap_stream) RAD_CUDA(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
  const long long epoch0 = alloc_epoch();
  RAD_CUDA(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal));
  g_sink = &w.g_sink_data;
  rad_status s = enqueue_pass(w, w.cap_stream);
  g_sink = nullptr;
  graph_undo_capture(w.g_sink_data);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(w.cap_stream, &graph);
  if (s != RAD_OK || e != cudaSuccess || alloc_epoch() != epoch0) {
    // failed, or a buffer moved while capturing: keep running eagerly
    if (graph) cudaGraphDestroy(graph);
    graph_release(w.g_sink_data);
    if (s != RAD_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    return RAD_OK;
  }
  e = cudaGraphInstantiate(&w.gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    w.gexec = nullptr;
    graph_release(w.g_sink_data);
    return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  w.g_prof = profiling_on();
  w.g_epoch = alloc_epoch();
  w.g_rois = w.rois;
  w.g_rd = w.rd;
  w.g_tuning = tuning();
  return RAD_OK;
}

// A graph stays valid while the ROI table, the diameter parameters, the
// tuning (kernel shapes), the profiling mode and every buffer are unchanged.
static bool graph_matches(const Work& w) {
  const rad_tuning_t& t = tuning();
  return w.gexec && w.g_epoch == alloc_epoch() && w.g_prof == profiling_on() && w.g_rois.size() == w.rois.size() &&
         same_bytes(w.g_rois.data(), w.rois.data(), sizeof(Roi) * w.rois.size()) && w.g_rd.size() == w.rd.size() &&
         same_bytes(w.g_rd.data(), w.rd.data(), sizeof(RoiDiam) * w.rd.size()) && same_bytes(&w.g_tuning, &t, sizeof(t));
}

rad_status status_from_dev(unsigned int st) {
  if (st & (DEV_ERR_VCAP | DEV_ERR_TCAP | DEV_ERR_CANDCAP | DEV_ERR_WORKCAP | DEV_ERR_PROBCAP)) {
    set_error("device pool too small (status 0x%x)", st);
    return RAD_ERR_CAPACITY;
  }
  if (st & DEV_ERR_TIMEOUT) {
    set_error("bounded device wait gave up (status 0x%x)", st);
    return RAD_ERR_TIMEOUT;
  }
  if (st) {
    set_error("device consistency check failed (status 0x%x)", st);
    return RAD_ERR_INTERNAL;
  }
  return RAD_OK;
}

static thread_local rad_call_stats_t g_stats;
static void record_stats(const ResultBlock& r, long long h2d, long long d2h, bool have_diam) {
  memset(&g_stats, 0, sizeof(g_stats));
  g_stats.h2d_bytes = h2d;
  g_stats.d2h_bytes = d2h;
  if (!have_diam) return;
  g_stats.problems = r.stats.problems;
  g_stats.tiles = r.stats.tiles;
  g_stats.tile_pairs = r.stats.tile_pairs;
  g_stats.work_items = r.stats.work_items;
  g_stats.items_evaluated = r.stats.items_evaluated;
  g_stats.pairs_evaluated = r.stats.pairs_evaluated;
  g_stats.candidates = r.stats.candidates;
  g_stats.coarse_pairs = r.stats.coarse_pairs;
}

// Whole pass on the prepared batch.  Capacities come from the previous call
// (the first call sizes them with a counting pass); an overflow is detected
// from the device status and the pass re-runs with grown pools.  From the
// second call on the same ROI table the pass is replayed as one CUDA graph
// (with per-kernel event pairs inside it when profiling is on).
static rad_status run_pass(Work& w, cudaStream_t st, bool use_graph, long long h2d_bytes) {
  if (w.vcap == 0) RAD_TRY(size_pools(w, st));
  for (int attempt = 0; attempt < 4; ++attempt) {
    bool replayed = false;
    if (use_graph && graph_matches(w)) {
      RAD_CUDA(cudaGraphLaunch(w.gexec, st));
      graph_replayed(w.g_sink_data);
      replayed = true;
    } else {
      RAD_TRY(enqueue_pass(w, st));
    }
    RAD_CUDA(cudaStreamSynchronize(st));
    if (replayed) graph_timed(w.g_sink_data);
    const ResultBlock& r = *w.host;
    const unsigned int s = r.stats.status | r.tot.status;
    if (r.tot.nv > w.vcap || r.tot.nt > w.tcap || (s & (DEV_ERR_VCAP | DEV_ERR_TCAP))) {
      w.drop_graph();
      RAD_TRY(size_pools(w, st));
      continue;
    }
    if (s & DEV_ERR_WORKCAP) { w.drop_graph(); w.ds.work_cap *= 4; continue; }
    if (s & DEV_ERR_CANDCAP) { w.drop_graph(); w.ds.cand_cap *= 4; continue; }
    RAD_TRY(status_from_dev(s));
    record_stats(r, h2d_bytes, (long long)(sizeof(ResultBlock) + sizeof(rad_features_t) * w.mb.n), true);
    if (use_graph && !graph_matches(w)) RAD_TRY(capture_pass(w));
    return RAD_OK;
  }
  return status_from_dev(w.host->stats.status | w.host->tot.status);
}

// Mesh only (rad_mesh / rad_soft_mesh / the soft adjoint): exact sizing, then
// vertices and triangles; the per-ROI results are read back.
static rad_status run_mesh_only(Work& w, cudaStream_t st, RoiOut* ro_host) {
  RAD_TRY(size_pools(w, st));
  RAD_TRY(enqueue_mesh(w, st, false));
  RAD_CUDA(cudaMemcpyAsync(w.host, w.dres(), sizeof(ResultBlock), cudaMemcpyDeviceToHost, st));
  if (ro_host) RAD_CUDA(cudaMemcpyAsync(ro_host, w.dro(), sizeof(RoiOut), cudaMemcpyDeviceToHost, st));
  RAD_CUDA(cudaStreamSynchronize(st));
  return status_from_dev(w.host->tot.status);
}

}  // namespace rad

struct rad_workspace {
  rad::Work work;
  rad_mesh_t mesh;
};

struct rad_batch {
  rad::Work work;
  int n = 0;
  std::vector<const void*> masks;
  std::vector<int64_t> dims;
  std::vector<double> spacing;
};

using namespace rad;

namespace {

rad_status check_geometry(const int64_t dims[3], const double spacing[3]) {
  if (!dims || !spacing) {
    set_error("dims and spacing must be non-NULL");
    return RAD_ERR_INVALID_ARG;
  }
  for (int k = 0; k < 3; ++k) {
    if (dims[k] < 1 || dims[k] > 16383) {
      set_error("dims[%d] = %lld outside [1, 16383]", k, (long long)dims[k]);
      return RAD_ERR_INVALID_ARG;
    }
    if (!(spacing[k] > 0.0) || !isfinite(spacing[k])) {
      set_error("spacing[%d] = %g must be finite and > 0", k, spacing[k]);
      return RAD_ERR_INVALID_ARG;
    }
  }
  // the packed grid of one mask is indexed with 32-bit arithmetic
  const long long words = (dims[1] + 3) * (dims[2] + 3) * ((dims[0] + 31) / 32);
  if (words >= (1LL << 31)) {
    set_error("mask of %lld x %lld x %lld voxels is too large (%lld packed words >= 2^31)", (long long)dims[0],
              (long long)dims[1], (long long)dims[2], words);
    return RAD_ERR_INVALID_ARG;
  }
  return RAD_OK;
}

rad_status check_device_ptr(const void* p, const char* what) {
  if (!p) {
    set_error("%s is NULL", what);
    return RAD_ERR_INVALID_ARG;
  }
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: cudaPointerGetAttributes failed: %s", what, cudaGetErrorString(e));
    return RAD_ERR_INVALID_ARG;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
    set_error("%s is not a device pointer", what);
    return RAD_ERR_INVALID_ARG;
  }
  return RAD_OK;
}

Work* work_of(rad_mesh_t* m) {
  if (!m->_priv) m->_priv = new Work();
  return static_cast<Work*>(m->_priv);
}

rad_workspace_t* ensure_ws(rad_workspace_t** ws) {
  if (!*ws) {
    *ws = new rad_workspace();
    memset(&(*ws)->mesh, 0, sizeof(rad_mesh_t));
  }
  return *ws;
}

// Marching cubes of one grid into the buffers of `w`, described in *mesh.
rad_status build_mesh(const void* data, bool soft, const int64_t dims[3], const double sp[3], Work& w,
                      rad_mesh_t* mesh, cudaStream_t st) {
  const void* ptrs[1] = {data};
  RAD_TRY(prepare(w, 1, ptrs, dims, sp, soft, st));
  RoiOut ro;
  RAD_TRY(run_mesh_only(w, st, &ro));
  mesh->n_vertices = ro.nv;
  mesh->n_triangles = ro.nt;
  mesh->n_voxels = ro.nvox;
  mesh->vtx_idx2 = w.idx2.as<int16_t>();
  mesh->vtx_t = soft ? w.vt.as<double>() : nullptr;
  mesh->tri = w.tri.as<int32_t>();
  mesh->mesh_volume = ro.vol6 / 6.0;
  mesh->surface_area = ro.area2 * 0.5;
  for (int k = 0; k < 3; ++k) {
    mesh->dims[k] = dims[k];
    mesh->spacing[k] = sp[k];
  }
  mesh->soft = soft ? 1 : 0;
  return RAD_OK;
}

rad_status check_mesh(const rad_mesh_t* mesh) {
  if (!mesh || !mesh->_priv) {
    set_error("mesh is NULL or was not built by rad_mesh / rad_soft_mesh");
    return RAD_ERR_INVALID_ARG;
  }
  return RAD_OK;
}

// Diameters of the mesh held by `w` (built by build_mesh on the same Work):
// variant 0 is the FP32-filter engine, RAD_FP64_EQUAL_LOAD ..
// RAD_FP64_PLAIN_1D the all-pairs FP64 kernels, RAD_FP64_CULLED the engine
// with FP64 pair evaluation.
rad_status shape_of_mesh(const rad_mesh_t* mesh, Work& w, int variant, rad_features_t* out, cudaStream_t st) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (variant >= RAD_FP64_EQUAL_LOAD && variant <= RAD_FP64_PLAIN_1D) {
      RAD_TRY(w.plain.reserve(sizeof(DiamResult)));
      RAD_TRY(enqueue_finish(w, false, st));
      if (mesh->n_vertices >= 2)
        RAD_TRY(diam_fp64_variant(variant, mesh->vtx_idx2, mesh->vtx_t, mesh->n_vertices, make_dims(mesh->dims),
                                  mesh->spacing, w.ds, w.plain.as<DiamResult>(), st));
      DiamResult pr;
      memset(&pr, 0, sizeof(pr));
      if (mesh->n_vertices >= 2)
        RAD_CUDA(cudaMemcpyAsync(&pr, w.plain.p, sizeof(DiamResult), cudaMemcpyDeviceToHost, st));
      RAD_CUDA(cudaStreamSynchronize(st));
      *out = w.hfeats[0];
      double* D[4] = {&out->Maximum3DDiameter, &out->Maximum2DDiameterSlice, &out->Maximum2DDiameterColumn,
                      &out->Maximum2DDiameterRow};
      int32_t* A[4] = {out->argmax3d, out->argmax_slice, out->argmax_column, out->argmax_row};
      for (int q = 0; q < 4; ++q) {
        const bool ok = mesh->n_vertices >= 2 && pr.i[q] >= 0;
        *D[q] = ok ? sqrt(pr.d2[q]) : 0.0;
        A[q][0] = ok ? pr.i[q] : -1;
        A[q][1] = ok ? pr.j[q] : -1;
      }
      record_stats(*w.host, 0, (long long)sizeof(DiamResult), false);
      return RAD_OK;
    }
    w.ds.fp64_pairs = variant == RAD_FP64_CULLED;
    const rad_status es = enqueue_shape(w, st);
    w.ds.fp64_pairs = false;
    RAD_TRY(es);
    RAD_TRY(enqueue_finish(w, true, st));
    RAD_CUDA(cudaStreamSynchronize(st));
    const unsigned int s = w.host->stats.status;
    if (s & DEV_ERR_WORKCAP) { w.ds.work_cap *= 4; continue; }
    if (s & DEV_ERR_CANDCAP) { w.ds.cand_cap *= 4; continue; }
    RAD_TRY(status_from_dev(s));
    *out = w.hfeats[0];
    record_stats(*w.host, 0, (long long)(sizeof(ResultBlock) + sizeof(rad_features_t)), true);
    return RAD_OK;
  }
  return status_from_dev(w.host->stats.status);
}

}  // namespace

extern "C" {

rad_status rad_mesh(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], rad_mesh_t* mesh,
                    void* stream) {
  RAD_TRY(check_geometry(dims, spacing));
  if (!mesh) { set_error("mesh is NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_device_ptr(mask_dev, "mask_dev"));
  return build_mesh(mask_dev, false, dims, spacing, *work_of(mesh), mesh, (cudaStream_t)stream);
}

rad_status rad_soft_mesh(const float* prob_dev, const int64_t dims[3], const double spacing[3], rad_mesh_t* mesh,
                         void* stream) {
  RAD_TRY(check_geometry(dims, spacing));
  if (!mesh) { set_error("mesh is NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_device_ptr(prob_dev, "prob_dev"));
  return build_mesh(prob_dev, true, dims, spacing, *work_of(mesh), mesh, (cudaStream_t)stream);
}

rad_status rad_shape(const rad_mesh_t* mesh, rad_features_t* out, void* stream) {
  RAD_TRY(check_mesh(mesh));
  if (!out) { set_error("out is NULL"); return RAD_ERR_INVALID_ARG; }
  return shape_of_mesh(mesh, *static_cast<Work*>(mesh->_priv), 0, out, (cudaStream_t)stream);
}

rad_status rad_shape_plain_fp64(const rad_mesh_t* mesh, rad_features_t* out, void* stream) {
  RAD_TRY(check_mesh(mesh));
  if (!out) { set_error("out is NULL"); return RAD_ERR_INVALID_ARG; }
  return shape_of_mesh(mesh, *static_cast<Work*>(mesh->_priv), RAD_FP64_PLAIN_1D, out, (cudaStream_t)stream);
}

rad_status rad_shape_fp64_variant(const rad_mesh_t* mesh, int variant, rad_features_t* out, void* stream) {
  RAD_TRY(check_mesh(mesh));
  if (!out) { set_error("out is NULL"); return RAD_ERR_INVALID_ARG; }
  if (variant < RAD_FP64_EQUAL_LOAD || variant > RAD_FP64_CULLED) {
    set_error("unknown FP64 diameter variant");
    return RAD_ERR_INVALID_ARG;
  }
  return shape_of_mesh(mesh, *static_cast<Work*>(mesh->_priv), variant, out, (cudaStream_t)stream);
}

rad_status rad_mesh_copy(const rad_mesh_t* mesh, int16_t* idx2, double* t, int32_t* tri, void* stream) {
  RAD_TRY(check_mesh(mesh));
  cudaStream_t st = (cudaStream_t)stream;
  if (idx2 && mesh->n_vertices)
    RAD_CUDA(cudaMemcpyAsync(idx2, mesh->vtx_idx2, sizeof(int16_t) * 3 * mesh->n_vertices, cudaMemcpyDefault, st));
  if (t && mesh->vtx_t && mesh->n_vertices)
    RAD_CUDA(cudaMemcpyAsync(t, mesh->vtx_t, sizeof(double) * mesh->n_vertices, cudaMemcpyDefault, st));
  if (tri && mesh->n_triangles)
    RAD_CUDA(cudaMemcpyAsync(tri, mesh->tri, sizeof(int32_t) * 3 * mesh->n_triangles, cudaMemcpyDefault, st));
  RAD_CUDA(cudaStreamSynchronize(st));
  return RAD_OK;
}

void rad_mesh_free(rad_mesh_t* mesh) {
  if (!mesh) return;
  delete static_cast<Work*>(mesh->_priv);
  memset(mesh, 0, sizeof(*mesh));
}

static rad_status extract_impl(const uint8_t* mask_dev, const int64_t dims[3], const double sp[3],
                               rad_features_t* out, rad_workspace_t* ws, cudaStream_t st, long long h2d_bytes) {
  Work& w = ws->work;
  const void* ptrs[1] = {mask_dev};
  RAD_TRY(prepare(w, 1, ptrs, dims, sp, false, st));
  RAD_TRY(run_pass(w, st, true, h2d_bytes));
  *out = w.hfeats[0];
  return RAD_OK;
}

rad_status rad_extract(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], rad_features_t* out,
                       rad_workspace_t** ws, void* stream) {
  RAD_TRY(check_geometry(dims, spacing));
  if (!out || !ws) { set_error("out and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_device_ptr(mask_dev, "mask_dev"));
  return extract_impl(mask_dev, dims, spacing, out, ensure_ws(ws), (cudaStream_t)stream, 0);
}

rad_status rad_extract_host(const uint8_t* mask_host, const int64_t dims[3], const double spacing[3],
                            rad_features_t* out, rad_workspace_t** ws, void* stream) {
  RAD_TRY(check_geometry(dims, spacing));
  if (!out || !ws || !mask_host) { set_error("mask_host, out and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  rad_workspace_t* w = ensure_ws(ws);
  const size_t bytes = (size_t)dims[0] * dims[1] * dims[2];
  // Pinned host memory is mapped into the device's address space: the
  // bit-packing kernel then reads the mask in place over the host link (one
  // pass, no staging copy).  Pageable memory is copied to a device buffer.
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, mask_host) == cudaSuccess && a.type == cudaMemoryTypeHost &&
      a.devicePointer != nullptr)
    return extract_impl(static_cast<const uint8_t*>(a.devicePointer), dims, spacing, out, w, (cudaStream_t)stream,
                        (long long)bytes);
  cudaGetLastError();  // pageable memory may report an error here
  RAD_TRY(w->work.mask.reserve(bytes));
  RAD_CUDA(cudaMemcpyAsync(w->work.mask.p, mask_host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  return extract_impl(w->work.mask.as<uint8_t>(), dims, spacing, out, w, (cudaStream_t)stream, (long long)bytes);
}

void rad_workspace_free(rad_workspace_t* ws) { delete ws; }

rad_status rad_batch_create(int n_rois, const uint8_t* const* masks_dev, const int64_t* dims, const double* spacing,
                            rad_batch_t** out, void* stream) {
  if (!out || !masks_dev || !dims || !spacing || n_rois < 1) {
    set_error("n_rois >= 1 and non-NULL masks_dev, dims, spacing, out required");
    return RAD_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_rois; ++i) {
    RAD_TRY(check_geometry(dims + 3 * i, spacing + 3 * i));
    RAD_TRY(check_device_ptr(masks_dev[i], "masks_dev[i]"));
  }
  rad_batch_t* b = new rad_batch();
  b->n = n_rois;
  b->masks.assign(masks_dev, masks_dev + n_rois);
  b->dims.assign(dims, dims + 3 * n_rois);
  b->spacing.assign(spacing, spacing + 3 * n_rois);
  cudaStream_t st = (cudaStream_t)stream;
  rad_status s = prepare(b->work, n_rois, b->masks.data(), dims, spacing, false, st);
  if (s == RAD_OK) s = run_pass(b->work, st, true, 0);  // sizes the pools and captures the graph
  if (s != RAD_OK) {
    delete b;
    return s;
  }
  *out = b;
  return RAD_OK;
}

rad_status rad_batch_run(rad_batch_t* b, rad_features_t* out, void* stream) {
  if (!b || !out) { set_error("batch and out must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  // re-plan (host only; uploads only if the tuning changed the parameters)
  RAD_TRY(prepare(b->work, b->n, b->masks.data(), b->dims.data(), b->spacing.data(), false, (cudaStream_t)stream));
  RAD_TRY(run_pass(b->work, (cudaStream_t)stream, true, 0));
  memcpy(out, b->work.hfeats, sizeof(rad_features_t) * b->n);
  return RAD_OK;
}

void rad_batch_destroy(rad_batch_t* b) { delete b; }

}  // extern "C"

namespace {

rad_status check_soft_args(int n, const float* const* probs, const int64_t* dims, const double* spacing) {
  if (n < 1 || !probs || !dims || !spacing) {
    set_error("n must be >= 1 and probs, dims, spacing non-NULL");
    return RAD_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    RAD_TRY(check_geometry(dims + 3 * i, spacing + 3 * i));
    RAD_TRY(check_device_ptr(probs[i], "prob_dev"));
  }
  return RAD_OK;
}

// Features of n soft maps: one pass (meshes, diameters, features), replayed
// as a CUDA graph when the same maps come again (the graph is captured on the
// second call with an unchanged map table, so a stream of new maps, as in
// training, never pays for captures it cannot reuse).
rad_status soft_features_impl(Work& w, int n, const float* const* probs, const int64_t* dims, const double* sp,
                              rad_features_t* out, cudaStream_t st) {
  std::vector<const void*> ptrs(probs, probs + n);
  RAD_TRY(prepare(w, n, ptrs.data(), dims, sp, true, st));
  const bool repeat = w.prev_rois.size() == w.rois.size() &&
                      same_bytes(w.prev_rois.data(), w.rois.data(), sizeof(Roi) * w.rois.size());
  w.prev_rois = w.rois;
  RAD_TRY(run_pass(w, st, repeat, 0));
  memcpy(out, w.hfeats, sizeof(rad_features_t) * n);
  return RAD_OK;
}

// Gradients of n soft maps: the meshes are recomputed and the adjoint runs
// right behind them, with one host synchronisation (pool sizes and argmax
// pairs are checked on the device; a pool overflow repeats the call's work).
rad_status soft_backward_impl(Work& w, int n, const float* const* probs, const int64_t* dims, const double* sp,
                              const double* gout, const int32_t* argmax, double* const* grads, cudaStream_t st) {
  std::vector<const void*> ptrs(probs, probs + n);
  RAD_TRY(prepare(w, n, ptrs.data(), dims, sp, true, st));
  std::vector<SoftMap>& maps = w.soft_maps_host;
  maps.resize(n);
  long long vox = 0;
  for (int i = 0; i < n; ++i) {
    SoftMap& m = maps[i];
    m.prob = probs[i];
    m.grad = grads[i];
    m.nx = (int)dims[3 * i]; m.ny = (int)dims[3 * i + 1]; m.nz = (int)dims[3 * i + 2]; m.pad = 0;
    m.sx = sp[3 * i]; m.sy = sp[3 * i + 1]; m.sz = sp[3 * i + 2];
    for (int k = 0; k < 6; ++k) m.gout[k] = gout[6 * i + k];
    for (int k = 0; k < 8; ++k) m.pair[k] = argmax[8 * i + k];
    m.vox0 = vox;
    vox += (long long)m.nx * m.ny * m.nz;
  }
  RAD_TRY(w.soft_maps.reserve(sizeof(SoftMap) * n));
  if (w.vcap == 0) RAD_TRY(size_pools(w, st));
  ResultBlock* dr = w.dres();
  for (int attempt = 0; attempt < 3; ++attempt) {
    RAD_TRY(w.gvtx.reserve(sizeof(double) * 3 * std::max<long long>(w.vcap, 1)));
    RAD_CUDA(cudaMemcpyAsync(w.soft_maps.p, maps.data(), sizeof(SoftMap) * n, cudaMemcpyHostToDevice, st));
    RAD_TRY(mesh_count(w.mb, w.ms, &dr->tot, w.dro(), st));
    RAD_TRY(mesh_emit(w.mb, w.ms, &dr->tot, w.dro(), w.idx2.as<int16_t>(), w.vt.as<double>(), w.tri.as<int32_t>(),
                      w.vcap, w.tcap, st));
    RAD_TRY(soft_adjoint(w.idx2.as<int16_t>(), w.vt.as<double>(), w.tri.as<int32_t>(), &dr->tot.nv, &dr->tot.nt,
                         w.vcap, w.tcap, w.dro(), w.soft_maps.as<SoftMap>(), n, vox, w.gvtx.as<double>(),
                         &dr->tot.status, st));
    RAD_CUDA(cudaMemcpyAsync(w.host, dr, sizeof(ResultBlock), cudaMemcpyDeviceToHost, st));
    RAD_CUDA(cudaStreamSynchronize(st));
    const MeshTotals& t = w.host->tot;
    if (t.nv > w.vcap || t.nt > w.tcap || (t.status & (DEV_ERR_VCAP | DEV_ERR_TCAP))) {
      RAD_TRY(size_pools(w, st));
      continue;
    }
    if (t.status & DEV_ERR_PAIR) {
      set_error("an argmax pair is not a vertex pair of its map's mesh");
      return RAD_ERR_INVALID_ARG;
    }
    record_stats(*w.host, 0, (long long)sizeof(ResultBlock), false);
    return status_from_dev(t.status);
  }
  return status_from_dev(w.host->tot.status);
}

}  // namespace

extern "C" {

rad_status rad_soft_forward(const float* prob_dev, const int64_t dims[3], const double spacing[3], double out[3],
                            int32_t argmax[2], rad_workspace_t** ws, void* stream) {
  if (!out || !argmax || !ws) { set_error("out, argmax and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_soft_args(1, &prob_dev, dims, spacing));
  rad_features_t f;
  RAD_TRY(soft_features_impl(ensure_ws(ws)->work, 1, &prob_dev, dims, spacing, &f, (cudaStream_t)stream));
  out[0] = f.SurfaceArea;
  out[1] = f.MeshVolume;
  out[2] = f.Maximum3DDiameter;
  argmax[0] = f.argmax3d[0];
  argmax[1] = f.argmax3d[1];
  return RAD_OK;
}

rad_status rad_soft_features(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                             rad_features_t* out, rad_workspace_t** ws, void* stream) {
  if (!out || !ws) { set_error("out and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_soft_args(1, &prob_dev, dims, spacing));
  return soft_features_impl(ensure_ws(ws)->work, 1, &prob_dev, dims, spacing, out, (cudaStream_t)stream);
}

rad_status rad_soft_batch_forward(int n, const float* const* probs_dev, const int64_t* dims, const double* spacing,
                                  rad_features_t* out, rad_workspace_t** ws, void* stream) {
  if (!out || !ws) { set_error("out and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_soft_args(n, probs_dev, dims, spacing));
  return soft_features_impl(ensure_ws(ws)->work, n, probs_dev, dims, spacing, out, (cudaStream_t)stream);
}

rad_status rad_soft_backward(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                             const double gout[3], const int32_t argmax[2], double* grad_dev, rad_workspace_t** ws,
                             void* stream) {
  if (!gout || !argmax || !ws) { set_error("gout, argmax and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_soft_args(1, &prob_dev, dims, spacing));
  RAD_TRY(check_device_ptr(grad_dev, "grad_dev"));
  const double g6[6] = {gout[0], gout[1], gout[2], 0.0, 0.0, 0.0};
  const int32_t a8[8] = {argmax[0], argmax[1], -1, -1, -1, -1, -1, -1};
  return soft_backward_impl(ensure_ws(ws)->work, 1, &prob_dev, dims, spacing, g6, a8, &grad_dev, (cudaStream_t)stream);
}

rad_status rad_soft_backward_planes(const float* prob_dev, const int64_t dims[3], const double spacing[3],
                                    const double gout[6], const int32_t argmax[8], double* grad_dev,
                                    rad_workspace_t** ws, void* stream) {
  if (!gout || !argmax || !ws) { set_error("gout, argmax and ws must be non-NULL"); return RAD_ERR_INVALID_ARG; }
  RAD_TRY(check_soft_args(1, &prob_dev, dims, spacing));
  RAD_TRY(check_device_ptr(grad_dev, "grad_dev"));
  return soft_backward_impl(ensure_ws(ws)->work, 1, &prob_dev, dims, spacing, gout, argmax, &grad_dev,
                            (cudaStream_t)stream);
}

rad_status rad_soft_batch_backward(int n, const float* const* probs_dev, const int64_t* dims, const double* spacing,
                                   const double* gout, const int32_t* argmax, double* const* grads_dev,
                                   rad_workspace_t** ws, void* stream) {
  if (!gout || !argmax || !grads_dev || !ws) {
    set_error("gout, argmax, grads_dev and ws must be non-NULL");
    return RAD_ERR_INVALID_ARG;
  }
  RAD_TRY(check_soft_args(n, probs_dev, dims, spacing));
  for (int i = 0; i < n; ++i) RAD_TRY(check_device_ptr(grads_dev[i], "grads_dev"));
  return soft_backward_impl(ensure_ws(ws)->work, n, probs_dev, dims, spacing, gout, argmax, grads_dev,
                            (cudaStream_t)stream);
}

rad_status rad_crop_resample(const uint8_t* mask_dev, const int64_t dims[3], const double spacing[3], int label,
                             int pad, const double new_spacing[3], uint8_t* out_dev, int64_t out_capacity,
                             int64_t out_dims[3], int64_t box_lo[3], double out_spacing[3], rad_workspace_t** ws,
                             void* stream) {
  RAD_TRY(check_geometry(dims, spacing));
  if (!out_dims || !box_lo || !out_spacing || !ws) {
    set_error("out_dims, box_lo, out_spacing and ws must be non-NULL");
    return RAD_ERR_INVALID_ARG;
  }
  if (label > 255 || pad < 0 || out_capacity < 0) {
    set_error("label must be < 256 (negative: any non-zero value), pad and out_capacity >= 0");
    return RAD_ERR_INVALID_ARG;
  }
  if (new_spacing)
    for (int k = 0; k < 3; ++k)
      if (!(new_spacing[k] > 0.0) || !std::isfinite(new_spacing[k])) {
        set_error("new_spacing must be positive and finite");
        return RAD_ERR_INVALID_ARG;
      }
  RAD_TRY(check_device_ptr(mask_dev, "mask_dev"));
  if ((dims[0] + 15) / 16 * dims[1] * dims[2] >= (1ll << 31)) {
    set_error("mask too large for one call (%lld 16-voxel chunks)", (long long)((dims[0] + 15) / 16 * dims[1] * dims[2]));
    return RAD_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Work& w = ensure_ws(ws)->work;
  PrepInfo info;
  RAD_TRY(prep_bbox(mask_dev, dims, spacing, label, pad, new_spacing, w.prep, &info, st));
  for (int k = 0; k < 3; ++k) {
    out_dims[k] = info.nout[k];
    box_lo[k] = info.lo[k];
    out_spacing[k] = new_spacing ? new_spacing[k] : spacing[k];
  }
  record_stats(ResultBlock{}, 0, (long long)sizeof(PrepInfo), false);
  if (info.empty) return RAD_OK;
  const long long need = info.nout[0] * info.nout[1] * info.nout[2];
  if ((info.nout[0] + 3) / 4 * info.nout[1] * info.nout[2] >= (1ll << 31)) {
    set_error("output of %lld voxels is too large for one call", need);
    return RAD_ERR_INVALID_ARG;
  }
  if (need > out_capacity || !out_dev) {
    set_error("output needs %lld bytes, capacity %lld", need, (long long)out_capacity);
    return RAD_ERR_CAPACITY;
  }
  RAD_TRY(check_device_ptr(out_dev, "out_dev"));
  return prep_gather(mask_dev, dims, spacing, label, new_spacing, info, w.prep, out_dev, st);
}

rad_status rad_check_bounded_wait(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf buf;
  RAD_TRY(buf.reserve(sizeof(ScanTile<1>) * 2 + 16));
  RAD_CUDA(cudaMemsetAsync(buf.p, 0, sizeof(ScanTile<1>) * 2 + 16, st));
  unsigned int* status = reinterpret_cast<unsigned int*>(buf.as<char>() + sizeof(ScanTile<1>) * 2);
  RAD_LAUNCH("wait_probe", rad::k_wait_probe, 1, 32, 0, st, buf.as<ScanTile<1>>(), status);
  unsigned int h = 0;
  RAD_CUDA(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st));
  RAD_CUDA(cudaStreamSynchronize(st));
  buf.release();
  if (h & DEV_ERR_TIMEOUT) {
    set_error("bounded device wait gave up as expected (status 0x%x)", h);
    return RAD_ERR_TIMEOUT;
  }
  set_error("bounded device wait did not report a timeout (status 0x%x)", h);
  return RAD_ERR_INTERNAL;
}

rad_status rad_set_tuning(const rad_tuning_t* set, rad_tuning_t* get) {
  if (set) {
    const bool ok_tile = set->tile == 64 || set->tile == 128 || set->tile == 256;
    const bool ok_thr = (set->tile == 64 && (set->threads == 64 || set->threads == 128)) ||
                        (set->tile == 128 && (set->threads == 64 || set->threads == 128 || set->threads == 256)) ||
                        (set->tile == 256 && (set->threads == 64 || set->threads == 128));
    if (!ok_tile || !ok_thr || set->ctas_per_sm < 1 || set->ctas_per_sm > 16 || set->cell_shift < 2 ||
        set->cell_shift > 7) {
      set_error("invalid tuning (tile %d, threads %d, ctas_per_sm %d, cell_shift %d)", set->tile, set->threads,
                set->ctas_per_sm, set->cell_shift);
      return RAD_ERR_INVALID_ARG;
    }
    g_tuning = *set;
  }
  if (get) *get = g_tuning;
  return RAD_OK;
}

rad_status rad_profile_enable(int on) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = on != 0;
  return RAD_OK;
}

int rad_profile_read(rad_kernel_stat_t* out, int cap) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  flush_pending(p);
  const int n = (int)p.stats.size();
  for (int i = 0; i < n && i < cap && out; ++i) out[i] = p.stats[i];
  return n;
}

void rad_profile_reset(void) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  flush_pending(p);
  for (auto& st : p.stats) {  // keep the entries: captured graphs refer to them
    st.launches = 0;
    st.total_ms = 0.0;
  }
}

int64_t rad_launch_count(void) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  return p.launches;
}

const char* rad_status_str(rad_status s) {
  switch (s) {
    case RAD_OK: return "RAD_OK";
    case RAD_ERR_INVALID_ARG: return "RAD_ERR_INVALID_ARG";
    case RAD_ERR_CUDA: return "RAD_ERR_CUDA";
    case RAD_ERR_CAPACITY: return "RAD_ERR_CAPACITY";
    case RAD_ERR_TIMEOUT: return "RAD_ERR_TIMEOUT";
    case RAD_ERR_OOM: return "RAD_ERR_OOM";
    case RAD_ERR_INTERNAL: return "RAD_ERR_INTERNAL";
  }
  return "RAD_ERR_UNKNOWN";
}

const char* rad_last_error(void) { return g_err; }

rad_status rad_last_call_stats(rad_call_stats_t* out) {
  if (!out) { set_error("out is NULL"); return RAD_ERR_INVALID_ARG; }
  *out = g_stats;
  return RAD_OK;
}

}  // extern "C"
