"""Benchmark: milliseconds per surface mesh of a 1,000,020-atom synthetic
assembly (60 icosahedrally arranged copies of a 16,667-atom globular unit on
a 250 A shell; D = 0.5, c = 1, precision 1e-3, min edge 0.25 A, 3 levels)
on one GB300, through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode mixed|fp64]
                  [--impl ours|reference]

One JSON line on rank 0.  `value` times mesh_gaussian_surface with the atoms
already resident in HBM and the mesh left on the device; `e2e` times
mesh_gaussian_surface_into with pinned host inputs and the mesh copied into
pinned host buffers kept across calls, copies included.  L2
is flushed (a 256 MB write) between timed steps, outside the timed region.
Under torchrun each rank meshes its own copy (replicas, weak scaling); the
reported time is the maximum over ranks.  --impl reference times the CPU
oracle on a bounded cut-out of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per surface mesh (1M atoms), mixed vs FP64 GPU; Gaussian evals/s, % peak"
WORKLOAD = dict(name="assembly1m", atoms=1000020, D=0.5, c=1.0, precision=1e-3, min_edge=0.25, max_depth=3)


def workload_desc(name):
    """The config string of a named workload (both arms report the same)."""
    params = "D=0.5, c=1, precision 1e-3, min edge 0.25 A, max_depth 3"
    if name == "assembly1m":
        return ("assembly1m: 1,000,020 atoms (60 x 16,667-atom globular unit on a 250 A icosahedral shell), "
                + params)
    if name.startswith("globular"):
        return "%s: %s-atom globular molecule (0.1 atoms/A^3), %s" % (name, name[len("globular"):], params)
    if name == "chain100":
        return "chain100: 100-atom random-walk chain, " + params
    return name
# plain-ALU peaks (FLOP/s) from the unit counts and clocks: 152 SMs at 2070 MHz;
# FP32: 128 FMA lanes/SM/clk; FP64: 2 FMA/SM/clk (1.25 TFLOP/s nominal);
# an FMA counts 2 flops
SM_COUNT, SM_MHZ = 152, 2070.0
PEAK_FP32 = SM_COUNT * 128 * 2 * SM_MHZ * 1e6
PEAK_FP64 = SM_COUNT * 2 * 2 * SM_MHZ * 1e6
# algorithmic work of one (cube, atom) term of the tensor accumulation:
# the rank-one update of the 4x4x4 tensor (64 FMA) and its 16 y-z products
FLOPS_PER_PAIR = 64 * 2 + 16
# DRAM bytes per cube of k_accum_f32: 394.7 MB for the 1,723,336 cubes of one
# launch in the ncu capture on the 20,000-atom molecule (writes of the 256 B
# tensor and 4 B bound per cube; atoms and cell list stay in L2)
ACCUM_F32_DRAM_BYTES_PER_CUBE = 394.7e6 / 1723336


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def job_ms(ms_local, ws, dist=None, device=None):
    """Replicas: every rank meshes its own copy in a step, so the job's step
    time is the slowest rank's and the whole-job time per mesh divides it by
    the ws meshes made.  Returns (step ms, ms per mesh)."""
    if ws > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_local = float(t.item())
    return ms_local, ms_local / ws


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "gs_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _batch_molecule(spec):
    import synth
    i, n, D = spec
    xyz, r = synth.globular(n, seed=1000 + i)
    return xyz, r, D


def make_batch_molecules(count=64):
    """The batch workload: 64 globular molecules, atom counts log-uniform in
    [500, 50000], D in {0.5, 0.9} (seeded)."""
    import multiprocessing as mp
    import synth
    specs = [(i, n, D) for i, (n, D) in enumerate(synth.batch_specs(count=count, seed=0))]
    with mp.get_context("spawn").Pool(processes=max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.map(_batch_molecule, specs, chunksize=1)


def cpu_baseline(cfg, half=6.0, margin=10.0, examined_full=None):
    """The oracle, as it stands, on a window of the workload: the atoms within
    `margin` of the cube of half-width `half` around the outermost atom of
    the first unit (the window's surface is the assembly's), meshed on every
    host core the oracle's threads can use.  The whole-mesh figure is an
    extrapolation, labelled as such: the window's time per examined cube
    times the examined cubes of the whole mesh (the GPU run's count when
    given).  The oracle scans every atom of its input for every cube, so the
    oracle run on the whole assembly at once would take longer still; this
    figure is what meshing it window by window would cost."""
    import oracle
    xyz, r = cfg["xyz"], cfg["r"]
    unit = xyz[:16667]
    cen = unit.mean(0)
    p0 = unit[np.argmax(((unit - cen) ** 2).sum(1))]
    sel = np.all((xyz >= p0 - half - margin) & (xyz <= p0 + half + margin), axis=1)
    sx, sr = np.ascontiguousarray(xyz[sel]), np.ascontiguousarray(r[sel])
    oracle.build()
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    m = oracle.mesh(sx, sr, cfg["D"], cfg["c"], cfg["precision"], cfg["min_edge"], cfg["max_depth"])
    dt = time.perf_counter() - t0
    ex_win = sum(m["stats"]["examined"])
    if examined_full is None:
        examined_full = len(r) / len(sr) * ex_win
    scale = examined_full / ex_win
    return {"value": dt * 1e3 * scale, "unit": "ms", "cores": threads, "kind": "oracle",
            "sample": "oracle.mesh (FP64, %d threads) on a window of the assembly: %d atoms within %.0f A of the "
                      "%.0f A cube around the outermost atom of unit 0 (%d examined cubes, %d triangles, %.1f s); "
                      "extrapolated x%.0f by examined cubes to the whole mesh (not measured)"
                      % (threads, len(sr), margin, 2 * half, ex_win, len(m["triangles"]), dt, scale),
            "sample_seconds": dt, "extrapolated": True}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import synth
    cfg = synth.config(WORKLOAD["name"])
    vals = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(cfg, half=args.ref_half)
        if i >= args.warmup:
            vals.append(b["value"])
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(WORKLOAD["name"]), "mode": "fp64 CPU oracle",
                       "parallelism": "single", "window_half_A": args.ref_half},
            "cpu_baseline": dict(b, value=v),
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def open_edges(tris):
    """Directed edges without exactly one oppositely oriented partner (0 for a
    closed, consistently oriented mesh)."""
    t = np.asarray(tris, dtype=np.int64)
    if len(t) == 0:
        return 0
    n = int(t.max()) + 1
    e = t[:, [0, 1, 1, 2, 2, 0]].reshape(-1, 2)
    fwd = e[:, 0] * n + e[:, 1]
    rev = e[:, 1] * n + e[:, 0]
    u, cnt = np.unique(fwd, return_counts=True)
    dup = int((cnt - 1).sum())
    return dup + int((~np.isin(rev, u)).sum())


READINGS = (("default: re-projected children, bounds first, sum norm, constrained values", {}),
            ("child re-expansion", {"child_mode": 1}),
            ("literal step-3 order", {"decision_order": 1}),
            ("max-norm precision test", {"precision_norm": 1}),
            ("euclidean-norm precision test", {"precision_norm": 2}),
            ("equal sizes across shared faces and edges", {"conform_mode": 1}))
# precisions at which the readings are compared; at 5e-2 cubes are accepted
# on two levels, where the readings for cubes of different sizes differ
READING_PRECISIONS = (1e-3, 1e-2, 5e-2)


def readings_form(gs, synth, torch, dev, stream, steps, barrier):
    cfg = synth.config("globular20k")
    x = torch.from_numpy(cfg["xyz"]).to(dev)
    r = torch.from_numpy(cfg["r"]).to(dev)
    out = {"workload": workload_desc("globular20k") + ", FP64 form; also at precisions 1e-2 and 5e-2, where "
                       "cubes are accepted above the finest level", "fidelity": "phi at triangle centroids"}
    rows = []
    for (label, kw), prec in [(rd, p) for p in READING_PRECISIONS for rd in READINGS]:
        args = (cfg["D"], cfg["c"], prec, cfg["max_depth"])
        ts = []
        for it in range(steps + 1):
            barrier()
            t0 = time.perf_counter()
            m = gs.mesh_gaussian_surface(x, r, *args, min_edge=cfg["min_edge"], stream=stream, device_output=True,
                                         **kw)
            torch.cuda.synchronize()
            if it > 0:
                ts.append((time.perf_counter() - t0) * 1e3)
        m = gs.mesh_gaussian_surface(x, r, *args, min_edge=cfg["min_edge"], stream=stream, **kw)
        st = m.stats
        cen = m.vertices[m.triangles].mean(1)
        phi = gs.gs_eval_field(cfg["xyz"], cfg["r"], cfg["D"], cfg["c"], cen, stream=stream)
        dev_rel = np.abs(phi - cfg["c"]) / cfg["c"]
        rows.append({"reading": label, "precision": prec, "ms_per_mesh": float(np.mean(ts)),
                     "ms_levels": st["ms_levels"], "accepted": st["accepted"][:cfg["max_depth"] + 1],
                     "pair_terms": st["pair_terms"], "examined": st["examined"][:cfg["max_depth"] + 1],
                     "n_cubes_final": st["n_cubes_final"], "n_triangles": st["n_triangles"],
                     "final_levels": np.bincount(np.asarray(m.cube_keys).astype(np.int64) >> 59,
                                                 minlength=cfg["max_depth"] + 1).tolist(),
                     "conformity_splits": st["conformity_splits"], "agreement_splits": st["agreement_splits"],
                     "constrained_vertices": st["constrained_vertices"], "loop_errors": st["loop_errors"],
                     "open_edges": open_edges(m.triangles),
                     "centroid_phi_err_max": float(dev_rel.max()) if len(dev_rel) else 0.0,
                     "centroid_phi_err_mean": float(dev_rel.mean()) if len(dev_rel) else 0.0})
    out["rows"] = rows
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="assembly1m")
    ap.add_argument("--ref-half", type=float, default=6.0, help="half-width (A) of the oracle's window")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-warmup", type=int, default=2, help="untimed end-to-end calls before the timed ones")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="timed end-to-end calls (host buffers, copies inside; at least 1)")
    ap.add_argument("--adaptive-steps", type=int, default=2,
                    help="mixed-form steps of the same assembly at precision 5e-2 (cubes on two levels)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="extra FP64-form steps timed for comparison")
    ap.add_argument("--diff-steps", type=int, default=2, help="differentiation-form steps (10k atoms) to time")
    ap.add_argument("--batch-steps", type=int, default=1, help="batch-form steps (64 molecules) to time")
    ap.add_argument("--readings-steps", type=int, default=1,
                    help="steps per alternative reading (20k atoms, FP64 form) timed and compared")
    args = ap.parse_args()
    args.e2e_steps = max(1, args.e2e_steps)   # the line's e2e needs one measured call
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    # batch-form molecules: generated on the host cores by a spawn pool before
    # any GPU call (the generator is a per-step Python random walk)
    batch_mols = None
    if args.batch_steps > 0 and rank == 0 and ws == 1:
        batch_mols = make_batch_molecules()

    import torch

    import paper_1611_03474_gb300 as gs
    import synth
    from paper_1611_03474_gb300 import build

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    cfg = synth.config(args.workload)
    mode = gs.GS_PREC_MIXED if args.mode == "mixed" else gs.GS_PREC_FP64
    stream = torch.cuda.current_stream()
    xyz_d = torch.from_numpy(cfg["xyz"]).to(dev)
    r_d = torch.from_numpy(cfg["r"]).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    kw = dict(min_edge=cfg["min_edge"], stream=stream)

    def run(x, r, prec, device_output=True):
        return gs.mesh_gaussian_surface(x, r, cfg["D"], cfg["c"], cfg["precision"], cfg["max_depth"],
                                        precision_mode=prec, device_output=device_output, **kw)

    for _ in range(args.warmup):
        run(xyz_d, r_d, mode)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times, stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m = run(xyz_d, r_d, mode)
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1))
        stats.append(m.stats)
    clk = clocks.stop()
    ms, ms_per_mesh = job_ms(float(np.mean(times)), ws, dist if ws > 1 else None, dev)

    # end to end: pinned host inputs, the whole mesh (vertices, triangles,
    # vertex and cube keys) copied into pinned host buffers that a serving
    # loop keeps across calls (allocated once, before the timed region, at
    # the sizes of the mesh above); both copies inside the timed region
    xyz_h = torch.from_numpy(cfg["xyz"]).pin_memory()
    r_h = torch.from_numpy(cfg["r"]).pin_memory()
    nv0, nt0, nc0 = m.n_vertices, m.n_triangles, m.n_cubes
    outs = (torch.empty((nv0, 3), dtype=torch.float64).pin_memory(),
            torch.empty((nt0, 3), dtype=torch.int32).pin_memory(),
            torch.empty(nv0, dtype=torch.int64).pin_memory(), torch.empty(nc0, dtype=torch.int64).pin_memory())
    e2e_times, e2e_stage = [], None
    for it in range(args.e2e_warmup + args.e2e_steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        nv, nt, nc, est = gs.mesh_gaussian_surface_into(xyz_h, r_h, cfg["D"], cfg["c"], cfg["precision"],
                                                        cfg["max_depth"], *outs, min_edge=cfg["min_edge"],
                                                        precision_mode=mode, stream=stream, stats=True)
        t1 = time.perf_counter()
        if it >= args.e2e_warmup:
            e2e_times.append((t1 - t0) * 1e3)
            e2e_stage = {k: est[k] for k in ("ms_total", "ms_upload", "ms_bin", "ms_levels", "ms_field",
                                             "ms_triangulate", "ms_weld", "ms_download")}
    nbytes_out = 24 * nv + 12 * nt + 8 * nv + 8 * nc
    # the mesh of the last end-to-end step, copied out of the buffers before
    # the link measurement below writes into them
    mh = types.SimpleNamespace(vertices=outs[0][:nv].numpy().copy(), triangles=outs[1][:nt].numpy().copy(),
                               vertex_keys=outs[2][:nv].numpy().view(np.uint64).copy(),
                               cube_keys=outs[3][:nc].numpy().view(np.uint64).copy())
    # the host link itself: one 1 GiB device-to-host copy into pinned memory
    # (best of 5), the bound on the end-to-end step's copies; and one copy of
    # the vertex array's size into the step's own pinned vertex buffer
    link = None
    try:
        vsrc = torch.empty(outs[0].numel(), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs[0].view(-1).copy_(vsrc, non_blocking=True)
        torch.cuda.synchronize()
        out_gbps = float(outs[0].numel() * 8 / (time.perf_counter() - t0) / 1e9)
        del vsrc
        src = torch.empty(1 << 28, dtype=torch.float32, device=dev)
        dst = torch.empty(1 << 28, dtype=torch.float32).pin_memory()
        bt = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            bt.append(time.perf_counter() - t0)
        link = {"d2h_GBps": float((1 << 30) / min(bt) / 1e9), "bytes": 1 << 30,
                "how": "torch copy of 1 GiB from device to pinned host memory, best of 5",
                "into_vertex_buffer_GBps": out_gbps}
        del src, dst
    except Exception as e:  # noqa: BLE001 (reported, not fatal)
        link = {"error": str(e)[:200]}
    e2e_ms = float(np.mean(e2e_times))

    # FP64 form for the comparison the metric names
    fp64 = None
    if args.fp64_steps > 0 and mode != gs.GS_PREC_FP64:
        ft = []
        for _ in range(args.fp64_steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mf = run(xyz_d, r_d, gs.GS_PREC_FP64)
            e1.record(stream)
            barrier()
            ft.append(e0.elapsed_time(e1))
        fp64 = {"ms_per_mesh": float(np.mean(ft)), "pair_terms": mf.stats["pair_terms"],
                "ms_accum": mf.stats["ms_accum"], "n_triangles": mf.stats["n_triangles"]}
        # FP32-vs-FP64 vertex error: the mixed mesh of the end-to-end step
        # against an (untimed) FP64 mesh with host outputs
        mfh = run(xyz_h, r_h, gs.GS_PREC_FP64, device_output=False)
        same = (np.array_equal(mh.vertex_keys, mfh.vertex_keys) and np.array_equal(mh.triangles, mfh.triangles)
                and np.array_equal(mh.cube_keys, mfh.cube_keys))
        fp64["same_cubes_and_topology"] = bool(same)
        fp64["max_vertex_diff_A"] = float(np.abs(mh.vertices - mfh.vertices).max()) if same else None
        del mfh

    # the adaptive path at full size: the same assembly in the same form at
    # precision 5e-2, where surface cubes are accepted on two levels and
    # cubes of different sizes join through constrained values
    adaptive = None
    if args.adaptive_steps > 0:
        at = []
        for it in range(args.adaptive_steps + 1):   # the first run warms up (pools, tuned launch shapes)
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ma = gs.mesh_gaussian_surface(xyz_d, r_d, cfg["D"], cfg["c"], 5e-2, cfg["max_depth"], precision_mode=mode,
                                          device_output=True, **kw)
            e1.record(stream)
            barrier()
            if it > 0:
                at.append(e0.elapsed_time(e1))
        sa = ma.stats
        adaptive = {"workload": workload_desc(args.workload).replace("precision 1e-3", "precision 5e-2"),
                    "mode": args.mode, "ms_per_mesh": float(np.mean(at)),
                    "accepted": sa["accepted"][:4], "forced": sa["forced"][:4], "examined": sa["examined"][:4],
                    "n_cubes_final": sa["n_cubes_final"], "n_triangles": sa["n_triangles"],
                    "constrained_vertices": sa["constrained_vertices"], "agreement_splits": sa["agreement_splits"],
                    "conformity_splits": sa["conformity_splits"], "mixed_cubes": sa["mixed_cubes"],
                    "loop_errors": sa["loop_errors"], "recheck_vertices": sa["recheck_vertices"],
                    "n_lattice_vertices": sa["n_lattice_vertices"], "vertex_terms": sa["vertex_terms"],
                    "vertex_mark_cubes": sa["vertex_mark_cubes"],
                    "stage_ms": {k: sa[k] for k in ("ms_levels", "ms_conformity",
                                                                                      "ms_field", "ms_triangulate",
                                                                                      "ms_weld")}}

    # differentiation form on the 10,000-atom globular molecule: forward mesh,
    # loss gradient per vertex, adjoint (gs_mesh_backward recomputes the mesh)
    diff = None
    if args.diff_steps > 0 and ws == 1:
        dcfg = synth.config("globular10k")
        dx, dr = dcfg["xyz"], dcfg["r"]
        tf, tb = [], []
        for it in range(args.diff_steps + 1):
            barrier()
            t0 = time.perf_counter()
            dm = gs.mesh_gaussian_surface(dx, dr, dcfg["D"], dcfg["c"], dcfg["precision"], dcfg["max_depth"],
                                          min_edge=dcfg["min_edge"], stream=stream)
            t1 = time.perf_counter()
            vol, area, gV, gA = gs.gs_volume_area(dm.vertices, dm.triangles, grad=True, stream=stream)
            gv = gV + gA
            t2 = time.perf_counter()
            gs.gs_mesh_backward(dx, dr, dcfg["D"], dcfg["c"], dcfg["precision"], dcfg["max_depth"], gv,
                                min_edge=dcfg["min_edge"], stream=stream)
            t3 = time.perf_counter()
            if it > 0:
                tf.append((t1 - t0) * 1e3)
                tb.append((t3 - t1) * 1e3)
        diff = {"workload": "globular10k: 10,000 atoms, D=0.5, c=1, L = volume + area, host buffers",
                "ms_forward": float(np.mean(tf)), "ms_backward": float(np.mean(tb)),
                "n_vertices": int(dm.vertices.shape[0]), "volume_A3": float(vol), "area_A2": float(area)}

    # batch form: 64 molecules in one call, with the shared level loop (each
    # level's kernels launched once over every molecule with the same D),
    # against whole meshes on 8 worker threads and one call at a time
    batch = None
    if batch_mols is not None:
        kwb = dict(precision_mode=mode, device_output=True)
        res = {}
        for label, nw, bmode in (("sequential", 1, gs.GS_BATCH_THREADS), ("threads", 8, gs.GS_BATCH_THREADS),
                                 ("shared_levels_w4", 4, gs.GS_BATCH_SHARED_LEVELS),
                                 ("shared_levels_w16", 16, gs.GS_BATCH_SHARED_LEVELS),
                                 ("shared_levels", 8, gs.GS_BATCH_SHARED_LEVELS)):
            ts = []
            for it in range(args.batch_steps + 1):
                flush.zero_()
                barrier()
                t0 = time.perf_counter()
                bm = gs.mesh_gaussian_surface_batch(batch_mols, cfg["c"], cfg["precision"], cfg["max_depth"],
                                                    n_workers=nw, batch_mode=bmode, **kwb)
                t1 = time.perf_counter()
                if it > 0:
                    ts.append((t1 - t0) * 1e3)
            res[label] = float(np.mean(ts))
            if label == "shared_levels":
                res["levels_ms"] = {}
                for (xyz_, r_, D_), m in zip(batch_mols, bm):
                    res["levels_ms"].setdefault("D=%g" % D_, float(m.stats["ms_levels"]))
        natoms = sum(len(m[1]) for m in batch_mols)
        batch = {"workload": "64 globular molecules, %d atoms in all, n log-uniform in [500, 50000], D in {0.5, 0.9}, "
                             "host inputs, device outputs" % natoms,
                 "ms_per_batch": res["shared_levels"], "ms_per_batch_threads": res["threads"],
                 "ms_per_batch_sequential": res["sequential"],
                 "ms_per_batch_by_workers": {"4": res["shared_levels_w4"], "8": res["shared_levels"],
                                             "16": res["shared_levels_w16"]},
                 "ms_level_loop_per_group": res["levels_ms"],
                 "molecules_per_s": 64 * 1e3 / res["shared_levels"], "n_workers": 8,
                 "n_triangles": int(sum(m.n_triangles for m in bm))}

    # the alternative readings of section 2.2 on the 20,000-atom globular
    # molecule, FP64 form: cube counts, work, time and mesh fidelity
    readings = None
    if args.readings_steps > 0 and ws == 1:
        readings = readings_form(gs, synth, torch, dev, stream, args.readings_steps, barrier)

    st = stats[-1]
    pairs = st["pair_terms"]
    acc_ms = float(np.mean([s["ms_accum"] for s in stats]))
    launches = max(1, st["n_accum_launches"])
    fp32 = mode == gs.GS_PREC_MIXED and st.get("recheck_cubes", 0) >= 0 and args.mode == "mixed"
    peak = PEAK_FP32 if fp32 else PEAK_FP64
    achieved = pairs * FLOPS_PER_PAIR / (acc_ms * 1e-3) if acc_ms > 0 else 0.0
    # DRAM traffic per launch: bytes per accumulated cube from the ncu capture
    # of the FP32 kernel on the 20,000-atom molecule (the kernel writes each
    # cube's tensor and bound and reads almost nothing), times the cubes one
    # launch accumulates here
    traffic = (ACCUM_F32_DRAM_BYTES_PER_CUBE * sum(st["examined"]) / launches) if fp32 else None
    roofline = {"bound": "alu", "kernel": "k_accum_f32" if fp32 else "k_accum_f64",
                "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch",
                "launches_per_step": launches, "ms_per_launch": acc_ms / launches,
                "peak_source": "152 SMs x 2070 MHz x (%s) FMA/SM/clk x 2 (unit counts and clocks)"
                               % ("128 FP32" if fp32 else "2 FP64")}
    evals = pairs + st["vertex_terms"]
    line = {
        "metric": METRIC, "value": ms_per_mesh, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "mode": args.mode, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "256 MB flush between timed steps"},
        "gaussian_evals_per_s": evals * ws / (ms * 1e-3),   # every rank evaluates its own replica
        "mesh": {"n_vertices": st["n_vertices"], "n_triangles": st["n_triangles"],
                 "n_cubes_final": st["n_cubes_final"], "examined": st["examined"][:4]},
        "stage_ms": {k: st[k] for k in ("ms_bin", "ms_levels", "ms_conformity", "ms_field", "ms_triangulate",
                                        "ms_weld")},
        "level_ms": st["ms_level"][:4],
        "recheck": {"cubes": st["recheck_cubes"], "vertices": st["recheck_vertices"],
                    "bounds": st["recheck_bounds"], "precision": st["recheck_precision"],
                    "zero": st["recheck_zero"], "rank": st["recheck_rank"],
                    "vertex_mark_cubes": st["vertex_mark_cubes"], "estimate_fast_cubes": st["estimate_fast_cubes"]},
        "pair_terms": pairs, "atom_octets": st["atom_octets"], "vertex_terms": st["vertex_terms"],
        "roofline": roofline,
        "clocks": clk,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(xyz_h.nbytes + r_h.nbytes),
                "d2h_bytes_per_step": int(nbytes_out), "runs": len(e2e_times), "warmup_runs": args.e2e_warmup,
                "min_ms": float(np.min(e2e_times)), "max_ms": float(np.max(e2e_times)),
                "copy_GBps_est": float(nbytes_out / ((e2e_ms - ms_per_mesh) * 1e-3) / 1e9)
                if e2e_ms > ms_per_mesh else None, "link": link, "stage_ms_last": e2e_stage,
                "buffers_pinned": {"inputs": bool(xyz_h.is_pinned() and r_h.is_pinned()),
                                   "outputs": bool(all(o.is_pinned() for o in outs)),
                                   # 1: the library sees page-locked memory mapped into the device
                                   "library_kind": [gs.memory_kind(b) for b in (xyz_h,) + outs]}},
        "gpu_launches": int(st["n_kernel_launches"]),
        # launch shapes the autotuner chose in this process (kernel, size class, choice, trial ms per shape)
        "autotune": gs.autotune_report(),
        "fp64_form": fp64,
        "adaptive_form": adaptive,
        "diff_form": diff,
        "batch_form": batch,
        "readings_form": readings,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, examined_full=sum(st["examined"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
