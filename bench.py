"""Benchmark of the shape-feature hot path on GB300.

Workload (one step): marching cubes + all shape features (mesh volume,
surface area, voxel volume, maximum 3D diameter and the three planar
diameters) of one 512x512x256 uint8 CT-shaped mask (3 rotated ellipsoids,
5 % boundary voxels flipped, spacing (0.7, 0.7, 2.5) mm), through the C ABI
entry point rad_extract with the mask resident in HBM.  The L2 (129 MB) is
flushed between steps by writing a 256 MB buffer (the mask itself is 67 MB).

Metric: diameter vertex-pairs/s = N (N - 1) / 2 / step time, whole job over
all ranks (replicas of the workload: the single-mask path does not shard).
Also reported: the plain FP64 all-pairs kernel on the same mesh, batched
crops per second, the end-to-end figure through host buffers, the roofline
of the dominant kernel and the FP64 CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "diameter vertex-pairs/s and batched ROIs/s vs plain FP64 kernel, 1 GB300, oracle-exact"
UNIT = "vertex-pairs/s"
WORKLOAD = ("ct_512x512x256: uint8 mask 512x512x256, spacing (0.7,0.7,2.5) mm, union of 3 rotated ellipsoids "
            "(semi-axes 60-150 voxels), 5% boundary voxels flipped, seed 0; mesh + all shape features per step")
FLOPS_PER_PAIR = 8  # 3 FADD + 1 FMUL + 2 FFMA (2 flops each) per evaluated pair
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def load_traffic(kernel):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + write.sum) from
    the committed ncu table profiles/dram_traffic.json, or None when the table
    has no entry for it or the kernel's source file changed since the counters
    were taken (its sha256 no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    entry = json.load(open(path)).get("kernels", {}).get(kernel)
    if not entry:
        return None
    src = os.path.join(ROOT, entry["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != entry["sha256_16"]:
        return None
    return int(entry["dram_bytes_read"]) + int(entry["dram_bytes_write"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = [r.split(",") for r in open(self.out.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend="nccl"):
    """Read the torchrun environment; for N > 1 join the process group (one
    rank per GPU; the ranks are independent replicas, the group only carries
    the barriers and the max over ranks of the step time)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif backend == "nccl" and torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Maximum of a per-rank float over all ranks (the whole-job step time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ms_max, world):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def kernel_work(name, ctx):
    """Algorithmic work of one launch of `name`: ("hbm", bytes) or ("alu", FP32 flops).

    Bytes count what the kernel must move at least once: the mask read and the
    bitset written (pack), the bitset read and the per-row counts written
    (count), the vertex and triangle output of the surface (emit: 18 B per
    vertex and 12 B per triangle), the vertices read and the sorted entries
    written (diameter sort).  Flops count the evaluated vertex pairs of the
    FP32 filter at 8 flops each."""
    nvox, words4, N, T, R = (ctx[k] for k in ("nvox", "bitset_bytes", "N", "T", "rows"))
    table = {
        "mc_pack_u8": nvox + words4,
        "mc_count": words4 + 16 * R,
        "mc_emit": 18 * N + 12 * T,
        "diam_hist": 6 * N,
        "diam_scatter": 6 * N + 4 * 20 * N,
    }
    if name == "diam_pairs_fp32":
        return "alu", FLOPS_PER_PAIR * ctx["pairs_evaluated"]
    if name in table:
        return "hbm", table[name]
    return None, None


MESH_KERNELS = ("mc_pack_u8", "mc_count", "mc_scan_rows", "mc_emit")


def mesh_stage_roofline(kernels, ctx, peak_gbs, steps):
    """The marching-cubes stage as a whole: mask in, vertices and triangles out
    (nvox + 18 N + 12 T bytes) over the summed per-kernel times of its kernels."""
    ms = sum(kernels[k]["total_ms"] for k in MESH_KERNELS if k in kernels) / steps
    if ms <= 0:
        return None
    b = ctx["nvox"] + 18 * ctx["N"] + 12 * ctx["T"]
    gbs = b / (ms / 1e3) / 1e9
    return {"kernels": list(MESH_KERNELS), "ms": ms, "algorithmic_bytes": b, "achieved": gbs, "peak": peak_gbs,
            "unit": "GB/s", "frac": gbs / peak_gbs}


def fp32_filter_entry(kernels, pairs_evaluated, derived_tflops, measured_tflops):
    """The FP32 filter's rate per launch (evaluated pairs x 8 flops over the
    pair kernel's mean launch time) against the derived and the measured
    FP32 peak; None when the pair kernel did not run."""
    kp = kernels.get("diam_pairs_fp32")
    if not kp or not kp.get("launches"):
        return None
    p_ms = kp["total_ms"] / kp["launches"]
    ach = pairs_evaluated * FLOPS_PER_PAIR / (p_ms / 1e3) / 1e12
    return {"kernel": "diam_pairs_fp32", "launch_ms": p_ms, "pairs_evaluated": pairs_evaluated,
            "flops_per_pair": FLOPS_PER_PAIR, "achieved_tflops": ach,
            "frac_of_derived": ach / derived_tflops, "derived_tflops": derived_tflops,
            "frac_of_measured": ach / measured_tflops, "measured_tflops": measured_tflops}


def timed(fn, steps, stream, flush):
    """Device milliseconds of fn() per call (CUDA events on `stream`, L2 flushed
    before each call) and host microseconds per call (wall clock)."""
    import torch
    dev_ms, host_us = [], []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        host_us.append((time.perf_counter() - t0) * 1e6)
        dev_ms.append(e0.elapsed_time(e1))
    return statistics.median(dev_ms), statistics.median(host_us)


def bench_ellipsoid32(args, stream, flush):
    """Per-ROI latency of a 32^3 ellipsoid through rad_extract (the pass
    replayed as one CUDA graph; results read back to the host every call)."""
    import torch
    from paper_2510_02894_gb300 import rad, synth
    m, sp = synth.ellipsoid_32(0)
    dev = torch.from_numpy(m).cuda()
    ws_new = rad.Workspace()
    t0 = time.perf_counter()
    rad.extract(dev, sp, ws_new)  # first call of a new workspace: allocation, tables from the cache
    first_us = (time.perf_counter() - t0) * 1e6
    ws = rad.Workspace()
    for _ in range(max(args.warmup, 3)):
        f = rad.extract(dev, sp, ws)
    launches0 = rad.launch_count()
    fbuf = rad.Features()
    dms, hus = timed(lambda: rad.extract(dev, sp, ws, out=fbuf), max(args.steps, 50), stream, flush)
    return {"workload": "ellipsoid_32: 32^3 uint8, semi-axes (10,7,5), spacing (1,1,1), seed 0",
            "n_vertices": f["n_vertices"], "latency_us": hus, "device_us": dms * 1e3,
            "first_call_new_workspace_us": first_us, "rois_per_s": 1e6 / hus,
            "gpu_launches_per_call": (rad.launch_count() - launches0) / max(args.steps, 50),
            "timing": "median of calls; host wall clock from the call to the features on the host"}


def bench_soft160(args, stream, flush, peak_gbs):
    """Soft 160^3 map: rad_soft_forward + rad_soft_backward per step."""
    import torch
    from paper_2510_02894_gb300 import rad, synth
    prob_np, sp = synth.soft_160(0)
    prob = torch.from_numpy(prob_np).cuda()
    grad = torch.empty(prob.shape, dtype=torch.float64, device="cuda")
    ws = rad.Workspace()
    gout = (1.0, 1.0, 1.0)
    box = {}

    def fwd():
        box["f"] = rad.soft_forward(prob, sp, ws)

    def bwd():
        rad.soft_backward(prob, sp, gout, box["f"][1], grad, ws)

    def both():
        fwd()
        bwd()
    for _ in range(max(args.warmup, 3)):
        both()
    steps = max(args.steps, 10)
    f_ms, _ = timed(fwd, steps, stream, flush)
    b_ms, _ = timed(bwd, steps, stream, flush)
    t_ms, t_us = timed(both, steps, stream, flush)
    nvox = prob.numel()
    algo = nvox * (4 + 4 + 8)  # forward reads 4 B/voxel; backward reads 4 B and writes the FP64 gradient
    gbs = algo / (t_ms / 1e3) / 1e9
    return {"workload": "soft_160: 160^3 float32 sigmoid(4 G_3(sd)) of a rotated ellipsoid, seed 0",
            "forward_ms": f_ms, "backward_ms": b_ms, "fwd_bwd_ms": t_ms, "fwd_bwd_host_us": t_us,
            "algorithmic_bytes": algo, "achieved_gbs": gbs, "hbm_frac": gbs / peak_gbs,
            "bytes_note": "4 B/voxel read (forward) + 4 B/voxel read + 8 B/voxel FP64 gradient written (backward)"}


def bench_blobs512x8(args, stream, flush):
    """8 x 512^3 blobs as one batch (one set of launches, replayed as one CUDA graph)."""
    import torch
    from paper_2510_02894_gb300 import rad, synth
    blobs = synth.blobs_512(0)
    devs = [torch.from_numpy(m).cuda() for m, _ in blobs]
    sps = [s for _, s in blobs]
    del blobs
    b = rad.Batch(devs, sps)
    feats = None
    for _ in range(max(args.warmup, 3)):
        feats = b.run()
    steps = max(min(args.steps, 10), 3)
    fbuf = b.features_buffer()
    ms, _ = timed(lambda: b.run(out=fbuf), steps, stream, flush)
    st = rad.last_call_stats()
    pairs = sum(f["n_vertices"] * (f["n_vertices"] - 1) / 2 for f in feats)
    out = {"workload": "blobs_512x8: 8 x 512^3 uint8 smoothed-noise blobs, ~40% filled, spacing (0.6,0.6,1.2), "
                       "seed 0", "rois": len(devs), "ms": ms, "rois_per_s": len(devs) / (ms / 1e3),
           "vertex_pairs_per_s": pairs / (ms / 1e3), "n_vertices": [f["n_vertices"] for f in feats],
           "pairs_evaluated_fp32": st["pairs_evaluated"], "voxels": int(sum(d.numel() for d in devs))}
    del b, devs
    torch.cuda.empty_cache()
    return out


def bench_prep(args, stream, flush, peak_gbs, dev, sp):
    """Crop of the CT mask to its ROI's box and nearest-neighbour resampling
    to 1 mm voxels (rad_crop_resample), the mask resident on the device."""
    from paper_2510_02894_gb300 import rad
    ws = rad.Workspace()
    out, lo, osp = rad.crop_resample(dev, sp, ws, new_spacing=(1.0, 1.0, 1.0))
    buf = out.reshape(-1).clone()
    for _ in range(max(args.warmup, 3)):
        rad.crop_resample(dev, sp, ws, new_spacing=(1.0, 1.0, 1.0), out=buf)
    ms, us = timed(lambda: rad.crop_resample(dev, sp, ws, new_spacing=(1.0, 1.0, 1.0), out=buf), max(args.steps, 10),
                   stream, flush)
    algo = dev.numel() + out.numel()  # the mask read once, the output written once
    gbs = algo / (ms / 1e3) / 1e9
    return {"workload": "ct_512x512x256 mask cropped to its ROI box and resampled to (1,1,1) mm",
            "out_dims_zyx": list(out.shape), "box_lo_xyz": list(lo), "ms": ms, "host_us": us,
            "algorithmic_bytes": algo, "achieved_gbs": gbs, "hbm_frac": gbs / peak_gbs,
            "note": "box reduction, index maps and gather kernels, with a host read of the box result (the output size) between the first and the others"}


def ablation_ct(m, ref, keys, stream):
    """The FP64 accumulation variants (rad_shape_fp64_variant 1-6) on one mesh:
    milliseconds per call and whether the results equal the FP32-filter engine's."""
    import torch
    from paper_2510_02894_gb300 import rad
    out = {}
    for name, v in rad.FP64_VARIANTS.items():
        rad.shape_fp64_variant(m, v)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = rad.shape_fp64_variant(m, v)
        e1.record(stream)
        e1.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "identical": all(f[k] == ref[k] for k in keys)}
    return out


def ablation_batch(crops, stream):
    """The same variants over the 256 crops, one mesh per crop (meshes built
    first, outside the timing): total milliseconds per variant."""
    import torch
    from paper_2510_02894_gb300 import rad
    meshes = [rad.mesh(torch.from_numpy(c).cuda(), sp) for c, sp in crops]
    keys = ("Maximum3DDiameter", "argmax3d", "Maximum2DDiameterSlice", "argmax_slice")
    base = [rad.shape(mm) for mm in meshes]
    out = {}
    for name, v in rad.FP64_VARIANTS.items():
        for mm in meshes[:4]:
            rad.shape_fp64_variant(mm, v)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [rad.shape_fp64_variant(mm, v) for mm in meshes]
        e1.record(stream)
        e1.synchronize()
        same = all(r[k] == b[k] for r, b in zip(res, base) for k in keys)
        out[name] = {"ms": e0.elapsed_time(e1), "identical": bool(same)}
    return out


def oracle_sample(mask, sp, n_slices, m_pairs_vertices):
    """Time the FP64 oracle as it stands on a bounded sample: its mesh on a
    central slab of z-slices (time scaled to all slices) and its brute-force
    diameter over the pairs of the slab's first vertices."""
    import oracle
    nz = mask.shape[0]
    z0 = max(0, nz // 2 - n_slices // 2)
    slab = np.ascontiguousarray(mask[z0:z0 + n_slices])
    t0 = time.perf_counter()
    om = oracle.OracleMesh(slab, sp)
    t_mesh = (time.perf_counter() - t0) * nz / slab.shape[0]
    src = om if om.nv >= m_pairs_vertices else oracle.OracleMesh(mask, sp)
    m = min(m_pairs_vertices, src.nv)
    t0 = time.perf_counter()
    oracle.diameters_bruteforce(src.u[:m], sp)
    t_pairs = time.perf_counter() - t0
    rate = m * (m - 1) / 2 / t_pairs
    return t_mesh, rate, oracle.num_threads(), m


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2510_02894_gb300 import synth
    mask, sp = synth.ct_512(0)
    N = oracle.OracleMesh(mask, sp).nv
    pairs = N * (N - 1) / 2
    vals, times = [], []
    for s in range(args.warmup + args.steps):
        t_mesh, rate, cores, m = oracle_sample(mask, sp, 16, 30000)
        full_s = t_mesh + pairs / rate
        if s >= args.warmup:
            vals.append(pairs / full_s)
            times.append(full_s * 1e3)
    value = statistics.mean(vals)
    sample = (f"per step: oracle mesh of 16 central of 256 z-slices (time scaled x16) + brute-force pairs of "
              f"{m} vertices ({m * (m - 1) // 2} pairs), extrapolated to N={N} ({pairs:.3e} pairs)")
    line = {"impl": "reference", "extrapolated": True, "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_vertices": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the 32^3, soft 160^3, 8 x 512^3 and crop lines")
    ap.add_argument("--configs", default="ellipsoid_32,soft_160,blobs_512x8,preprocess",
                    help="which of those lines to run (comma-separated subset of "
                         "ellipsoid_32,soft_160,blobs_512x8,preprocess)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the FP64 accumulation variants on the CT mesh and the 256 crops")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2510_02894_gb300 import autotune, rad, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    mask, sp = synth.ct_512(0)
    dev = torch.from_numpy(mask).cuda()
    pinned = torch.from_numpy(mask).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ws = rad.Workspace()
    ws_host = rad.Workspace()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        feats = rad.extract(dev, sp, ws)
        rad.extract_host(pinned.data_ptr(), mask.shape, sp, ws_host)
    stats = rad.last_call_stats()
    N, T = feats["n_vertices"], feats["n_triangles"]
    pairs = N * (N - 1) / 2
    tuned = {}
    tuning_default = rad.get_tuning()  # each workload's search starts from the library default
    if not args.no_autotune:  # pick tile / block shapes on this workload (a second or so)
        cache = os.path.join(tempfile.gettempdir(), "rad_bench_tuning.json")
        cfg, table = autotune.tune(lambda: rad.extract(dev, sp, ws), autotune.bucket(1, N), cache_path=cache)
        tuned["ct_512"] = {"config": cfg, "candidates": len(table),
                           "best_ms": min(ms for _, ms in table), "default_ms": table[0][1]}
    tuning_main = rad.get_tuning()

    # ---- timed region: device-resident inputs ------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    # the timed steps last a few ms, shorter than nvidia-smi's sampling period:
    # the same steps run untimed for about a second inside the sampling window
    # first, so the samples see the clocks under this load
    t_end = time.perf_counter() + 1.0
    fbuf = rad.Features()  # the call's rad_features_t, filled in place (no dict per step)
    while time.perf_counter() < t_end:
        flush.zero_()
        rad.extract(dev, sp, ws, out=fbuf)
    launches0 = rad.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    step_ms = []
    evaluated = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rad.extract(dev, sp, ws, out=fbuf)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        evaluated.append(rad.last_call_stats()["pairs_evaluated"])
    torch.cuda.synchronize()
    barrier(world)
    launches = rad.launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), world)
    value = job_throughput(pairs, ms, world)

    # ---- per-kernel durations: the same steps with CUDA events around every
    # kernel (event-record nodes inside the replayed graph) --------------------
    rad.profile_enable(True)
    rad.extract(dev, sp, ws)  # re-capture with the event nodes
    rad.profile_reset()
    prof_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rad.extract(dev, sp, ws, out=fbuf)
        e1.record(stream)
        e1.synchronize()
        prof_ms.append(e0.elapsed_time(e1))
    rad.profile_enable(False)
    prof = rad.profile_read()
    rad.extract(dev, sp, ws)  # back to the graph without event nodes

    # ---- end to end through host buffers ------------------------------------------
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rad.extract_host(pinned.data_ptr(), mask.shape, sp, ws_host, out=fbuf)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    hstats = rad.last_call_stats()
    e2e = max_over_ranks(statistics.mean(e2e_ms), world)

    # ---- roofline of the dominant kernel ---------------------------------------------
    peaks, peak_kind = load_peaks()
    props = torch.cuda.get_device_properties(local)
    sm_max = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
    fp32_peak_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    d = dict(nvox=int(mask.size), N=N, T=T, rows=(mask.shape[1] + 1) * (mask.shape[0] + 1),
             words_per_row=(mask.shape[2] + 31) // 32,
             bitset_bytes=4 * ((mask.shape[2] + 31) // 32) * (mask.shape[1] + 3) * (mask.shape[0] + 3),
             cubes=stats.get("cubes", T // 2), pairs_evaluated=statistics.mean(evaluated))
    kernels = {k: v for k, v in prof.items() if v["launches"] > 0}
    total_ms = sum(v["total_ms"] for v in kernels.values()) or 1.0
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    bound, amount = kernel_work(dom, d)
    per_launch_ms = kernels[dom]["total_ms"] / kernels[dom]["launches"]
    roof = {"kernel": dom, "share": kernels[dom]["total_ms"] / total_ms, "launch_ms": per_launch_ms}
    if bound == "hbm":
        ach = amount / (per_launch_ms / 1e3) / 1e9
        roof.update({"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / peaks["hbm_gbs"], "traffic": load_traffic(dom), "peak_source": peak_kind,
                     "algorithmic_bytes": amount})
    elif bound == "alu":
        ach = amount / (per_launch_ms / 1e3) / 1e12
        roof.update({"bound": "alu", "achieved": ach, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                     "frac": ach / fp32_peak_tflops, "traffic": load_traffic(dom),
                     "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "algorithmic_flops": amount})
    else:
        roof.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
    # ---- measured multiply-add peaks (outside every timed region) -------------------
    probe = {"fp32_tflops": rad.peak_probe(rad.PROBE_FP32), "fp32x2_tflops": rad.peak_probe(rad.PROBE_FP32X2),
             "fp64_tflops": rad.peak_probe(rad.PROBE_FP64),
             "how": "rad_peak_probe: one wave of 256-thread blocks, 8 independent multiply-add chains per thread "
                    "in registers, second of two launches timed with CUDA events; 2 flops per fma"}
    fp32_measured = max(probe["fp32_tflops"], probe["fp32x2_tflops"])
    fp32_filter = fp32_filter_entry(kernels, d["pairs_evaluated"], fp32_peak_tflops, fp32_measured)
    if roof.get("bound") == "alu":
        roof["peak_measured"] = fp32_measured
    kernel_table = {k: {"launches_per_step": v["launches"] / args.steps, "ms_per_step": v["total_ms"] / args.steps,
                        "share": v["total_ms"] / total_ms} for k, v in sorted(kernels.items(),
                                                                              key=lambda kv: -kv[1]["total_ms"])}

    # ---- plain FP64 all-pairs kernel on the same mesh -------------------------------
    plain = None
    if not args.no_plain:
        m = rad.mesh(dev, sp)
        rad.shape(m)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fp = rad.shape_plain_fp64(m)
        e1.record(stream)
        e1.synchronize()
        pms = e0.elapsed_time(e1)
        e0.record(stream)
        ff = rad.shape(m)
        e1.record(stream)
        e1.synchronize()
        fms = e0.elapsed_time(e1)
        keys = ("Maximum3DDiameter", "Maximum2DDiameterSlice", "Maximum2DDiameterColumn", "Maximum2DDiameterRow",
                "argmax3d", "argmax_slice", "argmax_column", "argmax_row")
        for _ in range(3):
            rad.shape_fp64_variant(m, rad.FP64_CULLED)
        e0.record(stream)
        fc = rad.shape_fp64_variant(m, rad.FP64_CULLED)
        e1.record(stream)
        e1.synchronize()
        cms = e0.elapsed_time(e1)
        cstats = rad.last_call_stats()
        same = all(fp[k] == ff[k] and fc[k] == ff[k] for k in keys)
        plain = {"ms": pms, "pairs_per_s": pairs / (pms / 1e3), "fp32_filter_shape_ms": fms,
                 "culled_fp64_shape_ms": cms, "culled_fp64_pairs_evaluated": cstats["pairs_evaluated"],
                 "speedup_vs_plain": pms / fms, "fp32_filter_speedup_vs_culled_fp64": cms / fms,
                 "identical_results": bool(same),
                 "fp64_flops_per_pair": 11, "fp64_tflops": pairs / (pms / 1e3) * 11 / 1e12,
                 "fp64_frac_of_measured": pairs / (pms / 1e3) * 11 / 1e12 / probe["fp64_tflops"],
                 "note": "plain = all pairs in FP64; culled_fp64 = the same tile walk and culling as the FP32 "
                         "filter, every surviving pair in FP64; shape timings from a built mesh (rad_shape)"}
        if args.ablation:
            plain["ablation"] = ablation_ct(m, ff, keys, stream)

    # ---- batched crops: 256 ROIs in one set of launches (one CUDA graph) -----------
    batch = None
    if not args.no_batch:
        crops = synth.batch_256(0)
        devs = [torch.from_numpy(c).cuda() for c, _ in crops]
        b = rad.Batch(devs, [s for _, s in crops])
        if not args.no_autotune:
            rad.set_tuning(**tuning_default)
            nb = sum(f["n_vertices"] for f in b.run())
            cache = os.path.join(tempfile.gettempdir(), "rad_bench_tuning.json")
            cfg, table = autotune.tune(b.run, autotune.bucket(len(devs), nb), cache_path=cache)
            tuned["batch_256"] = {"config": cfg, "candidates": len(table),
                                  "best_ms": min(ms for _, ms in table), "default_ms": table[0][1]}
        bbuf = b.features_buffer()  # rad_features_t per ROI, filled in place by each call
        for _ in range(args.warmup):
            b.run(out=bbuf)
        bms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(out=bbuf)
            e1.record(stream)
            e1.synchronize()
            bms.append(e0.elapsed_time(e1))
        t0 = time.perf_counter()
        [f.as_dict() for f in bbuf]  # the binding's optional conversion to Python dicts, timed on its own
        dicts_ms = (time.perf_counter() - t0) * 1e3
        bs = rad.last_call_stats()
        bm = statistics.mean(bms)
        # per-kernel durations of the batch (event nodes in its graph)
        rad.profile_enable(True)
        b.run()
        rad.profile_reset()
        for _ in range(args.steps):
            flush.zero_()
            b.run()
        torch.cuda.synchronize()
        rad.profile_enable(False)
        bprof = {k: v for k, v in rad.profile_read().items() if v["launches"] > 0}
        b.run()
        btot = sum(v["total_ms"] for v in bprof.values()) or 1.0
        batch_kernels = {k: {"ms_per_run": v["total_ms"] / args.steps, "share": v["total_ms"] / btot}
                         for k, v in sorted(bprof.items(), key=lambda kv: -kv[1]["total_ms"])}
        total_pairs = sum(f["n_vertices"] * (f["n_vertices"] - 1) / 2 for f in b.run())
        batch = {"rois": len(devs), "ms": bm, "rois_per_s": len(devs) / (bm / 1e3),
                 "vertex_pairs_per_s": total_pairs / (bm / 1e3), "voxels": int(sum(c.size for c, _ in crops)),
                 "mode": "rad_batch_run: one launch per stage over all 256 ROIs, replayed as one CUDA graph; "
                         "features returned as rad_features_t in host memory",
                 "python_dicts_ms": dicts_ms,
                 "pairs_evaluated_fp32": bs["pairs_evaluated"], "tuning": rad.get_tuning(),
                 "diam_stats": bs, "kernels": batch_kernels}
        if args.ablation:
            batch["ablation"] = ablation_batch(crops, stream)
        rad.set_tuning(**tuning_main)

    # ---- the other workloads: 32^3 latency, soft 160^3 forward + adjoint, 8 x 512^3 batch ----
    configs = {}
    if not args.no_configs:
        want = set(c.strip() for c in args.configs.split(","))
        if "ellipsoid_32" in want:
            configs["ellipsoid_32"] = bench_ellipsoid32(args, stream, flush)
        if "soft_160" in want:
            configs["soft_160"] = bench_soft160(args, stream, flush, peaks["hbm_gbs"])
        if "blobs_512x8" in want:
            configs["blobs_512x8"] = bench_blobs512x8(args, stream, flush)
        if "preprocess" in want:
            configs["preprocess"] = bench_prep(args, stream, flush, peaks["hbm_gbs"], dev, sp)

    # ---- CPU baseline: the oracle on a bounded sample --------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_mesh, rate, cores, m = oracle_sample(mask, sp, 16, 60000)
        full_s = t_mesh + pairs / rate
        cpu = {"value": pairs / full_s, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": True,
               "sample": (f"oracle mesh of 16 central of 256 z-slices (time x16) + FP64 brute-force pairs of {m} "
                          f"vertices, extrapolated to all {pairs:.3e} pairs (mesh {t_mesh:.2f} s, "
                          f"{rate:.3e} pairs/s)")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8+f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_vertices": N, "n_triangles": T, "pairs": pairs,
                           "pairs_evaluated_fp32": d["pairs_evaluated"], "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world}", "diam_stats": stats, "tuning": tuning_main,
                           "autotune": tuned},
                "roofline": roof, "mesh_stage": mesh_stage_roofline(kernels, d, peaks["hbm_gbs"], args.steps),
                "fp32_filter": fp32_filter, "peaks_probe": probe,
                "kernels": kernel_table, "ms_per_step_with_kernel_events": statistics.mean(prof_ms),
                "e2e": {"value": job_throughput(pairs, e2e, world), "unit": UNIT, "ms_per_step": e2e,
                        "h2d_bytes_per_step": hstats["h2d_bytes"], "d2h_bytes_per_step": hstats["d2h_bytes"]},
                "plain_fp64": plain, "batched": batch, "configs": configs, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
