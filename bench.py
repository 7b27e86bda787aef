#!/usr/bin/env python
"""Throughput of Hamiltonian integration + density update on one GB300 (points/s).

One step = nao_integrate_h (evaluate phi, grad phi per batch; h[B] contraction; scatter into
H; mirror) followed by nao_update_density (evaluate phi; density contraction; N_e) over the
whole grid, inputs resident in device memory. The default workload is the 375-atom
two-species slab (15,000 basis functions, 80 x 434 points per atom = 13,020,000 points,
batches <= 200 points; the stand-in for the paper's Bi2Se3 slab of Sec. 4), on the split
path at the slice count whose accuracy the full-size parity test checks on the same input.
``--config 1`` times the 64-atom diamond-lattice cluster instead. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|fp64|fp32] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own
GPU (the path has no exchange step on one handle); the line reports all ranks' points
divided by the slowest rank's time. ``--impl reference`` times the FP64 CPU oracle on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hamiltonian integration + density update pts/s, split-prec vs FP64; p99 latency"
WORKLOADS = {
    1: ("diamond64: 64-atom diamond-lattice cluster (cubic cell 10.26 bohr), 1600 basis functions "
        "(2s2p2d1f per atom), 60x306 points per atom = 1,175,040 points, batches <= 300 points"),
    2: ("slab375: 375-atom layered slab of two species (150 A : 225 B, 15 layers of 5x5, a = 7.8 bohr, "
        "pitch 3.5 bohr), 15,000 basis functions (4s3p4d1f per atom), 80x434 points per atom = "
        "13,020,000 points, batches <= 200 points"),
}
# split slices timed per workload: the count whose e <= 1e-10 the full-size parity tests check
# on the same input (tests/test_gpu_slab.py, tests/test_gpu_fullsize.py)
BENCH_SLICES = {1: 11, 2: 11}
# digit format timed per workload (bf16: base-64 digits, kind::f16; e4m3: base-32 digits,
# kind::f8f6f4) and the slice counts of each format that the parity tests check
BENCH_DIGITS = {1: "e4m3", 2: "e4m3"}
BENCH_SLICES_E4M3 = {1: 14, 2: 14}
# the split setting of the grouped and serving blocks (the molecule tests check it)
BENCH_SPLIT_OPTS = {"split_slices": 14, "split_digits": 1}
BENCH_SERVE_OPTS = {"split_slices": 14, "split_digits": 1}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=[None, "fp64", "fp32", "split"])
    ap.add_argument("--config", type=int, default=2, choices=[0, 1, 2],
                    help="workload: 2 = slab375 (default), 1 = diamond64, 0 = the 3-atom molecule")
    ap.add_argument("--cells", type=int, default=2,
                    help="diamond cluster: cubic cells per edge (2 = the 64-atom workload; 1 = an 8-atom case "
                         "for profiling captures, not a bench line)")
    ap.add_argument("--slab-layers", type=int, default=15,
                    help="slab: layers (15 = the 375-atom workload; fewer = a profiling case, not a bench line)")
    ap.add_argument("--scratch-mb", type=int, default=0,
                    help="evaluation scratch of the handle in MiB (0: the library default; the split slices get twice this)")
    ap.add_argument("--digits", default=None, choices=[None, "bf16", "e4m3"],
                    help="split path digit format (default: the one the workload is benched with)")
    ap.add_argument("--slices", type=int, default=None,
                    help="split path: slices per operand (default: the count the full-size parity test checks "
                         "on the workload; the library default is 12)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target single-thread CPU time of the oracle baseline's sample (its size is calibrated)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precisions")
    ap.add_argument("--serve-requests", type=int, default=120,
                    help="requests of the serving stream (Poisson arrivals at 200/s, 3-200 atoms)")
    ap.add_argument("--serve-fp64-requests", type=int, default=24,
                    help="the first requests of the same stream run again on the FP64 path")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic-silicon measurement")
    ap.add_argument("--grouped-molecules", type=int, default=128,
                    help="molecules of the batching configuration on their species' grids (0 skips it; "
                         "the stated configuration is 1024)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}




def alu_peak(kind: str):
    """FP64 or FP32 FMA throughput measured on this machine (profiles/peaks_fp64_fp32_dmma.txt)."""
    key = {"fp64": "fp64_fma_tflops", "fp32": "fp32_fma_tflops"}[kind]
    path = os.path.join(ROOT, "profiles", "peaks_fp64_fp32_dmma.txt")
    try:
        for line in open(path):
            if line.startswith(key):
                return float(line.split()[1]), "measured FMA loop (profiles/peaks_fp64_fp32_dmma.txt)"
    except Exception:
        pass
    return ({"fp64": 1.25, "fp32": 80.0}[kind], "nominal")


SERVE_GRID = dict(n_rad=30, n_theta=8, n_phi=9)


def serving(n_requests: int, device: int, fp64_requests: int) -> dict:
    """The request stream through the continuous-batching loop: every request on the split path,
    then the first fp64_requests of the same stream (same arrival times) on the FP64 path."""
    from paper_1912_06636_gb300 import serve, synth

    stream = synth.serving_stream(n_requests, rate=200.0, seed=4, n_min=3, n_max=200)
    t0 = time.perf_counter()
    reqs = []
    for rid, (t, na, seed) in enumerate(stream):
        s = synth.random_molecule(na, seed, **SERVE_GRID)
        reqs.append(serve.Request(rid=rid, system=s, v0=s.potential(on_device=True), arrival_s=t, n_iter=20, seed=seed))
    gen_s = time.perf_counter() - t0
    out = {"workload": f"{n_requests} requests, Poisson arrivals at 200/s (seed 4), molecules of 3-200 atoms "
                       f"(log-uniform; species Si/A/B), {SERVE_GRID['n_rad']}x{SERVE_GRID['n_theta'] * SERVE_GRID['n_phi']} "
                       "points per atom, batches <= 200 points, 20 iterations each (v perturbed 1%, fresh P), "
                       f"HBM budget 150 GB, 16 slots, CUDA graphs; FP64 on the first {min(fp64_requests, n_requests)} "
                       "requests of the same stream",
           "atoms_mean": float(sum(na for _, na, _ in stream) / max(len(stream), 1)),
           "points_total": int(sum(len(r.v0) for r in reqs)), "generate_s": gen_s}
    for prec, rs in (("split", reqs), ("fp64", reqs[:fp64_requests])):
        if not rs:
            continue
        srv = serve.Server(prec=prec, hbm_budget_bytes=150 << 30, max_active=16, device=device, **BENCH_SERVE_OPTS)
        res = srv.run(rs)
        sm = serve.summarize(res, srv.stats)
        # the rate the server sustains while requests wait: requests over the busy period
        busy = max(r.done_s for r in res) - min(r.admitted_s for r in res)
        sm["sustainable_requests_per_s"] = len(res) / busy if busy > 0 else None
        sm["arrival_rate_per_s"] = 200.0
        out[prec] = sm
    if "fp64" in out:
        # the same requests on both paths: the prefix the FP64 run served
        k = out["fp64"]["requests"]
        split_prefix = serve.Server(prec="split", hbm_budget_bytes=150 << 30, max_active=16, device=device,
                                    **BENCH_SERVE_OPTS)
        res = split_prefix.run(reqs[:k])
        pre = serve.summarize(res, split_prefix.stats)
        out["split_on_fp64_prefix"] = {"requests": k, "p50_ms": pre["p50_ms"], "p99_ms": pre["p99_ms"],
                                       "makespan_s": pre["makespan_s"]}
        if pre["p99_ms"] and out["fp64"]["p99_ms"]:
            out["p99_speedup_vs_fp64"] = out["fp64"]["p99_ms"] / pre["p99_ms"]
    return out


# DRAM bytes per algorithmic FLOP_H of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the captured launches / their FLOP_H): the
# FP64 contraction on the 8-atom profiling case (a launch's traffic grows with tiles x K, i.e. with
# FLOP_H). Valid only for the kernel version and slice count the capture was taken with.
TRAFFIC_PER_FLOP_H = {
    (1, "h_fp64", 0): ((359.834112e6 + 3.945472e6) / 4.6096304e9, "profiles/h_simt_kernel_diamond8_fp64.md"),
}
# DRAM bytes per issued tensor FLOP of the split H contraction, from one ncu capture of one launch
# of the 125-atom slab (the first five layers of the 375-atom workload, the same batch shapes):
# dram__bytes_read.sum + dram__bytes_write.sum over sm__ops_path_tensor_op_utcqmma_src_fp8_dst_fp32
# (the slices are read from DRAM once and re-read from L2, so the traffic grows with the tiles
# issued). Scaled by the issued FLOP of this run's average launch. Valid only for the kernel
# version, digit format and slice count the capture was taken with (e4m3, 14 slices).
TRAFFIC_PER_ISSUED_FLOP = {
    (2, "h_split", 14): ((1.044792e9 + 5.37984e6) / 2.6126843904e12, "profiles/h_tc_kernel_slab125_e4m3.md"),
}


def grouped(n_mol: int, device: int, steps: int = 3, per_molecule_max: int = 256) -> dict:
    """Many molecules (the batching configuration): molecules of 3-60 atoms on their species'
    grids with batch sizes log-uniform in [20, 400], in one grouped handle (one launch per kernel
    for all of them, CUDA graphs), the H + n step timed on the split path (library default
    slices) and on the FP64 path; against one handle per molecule (created one after the other,
    each step timed on its own and summed) when there are at most per_molecule_max of them
    (creating a thousand handles would dominate the run)."""
    import numpy as np
    import torch

    from paper_1912_06636_gb300 import nao, synth

    t0 = time.perf_counter()
    systems, bs = synth.molecule_set(n_mol, seed=3000, n_min=3, n_max=60, b_min=20, b_max=400, species_grids=True)
    dev = torch.device("cuda", device)
    vs = [torch.from_numpy(s.potential(on_device=True)).to(dev) for s in systems]
    Ps = [torch.from_numpy(synth.density_matrix(s, 3000 + k, rank=64)).to(dev) for k, s in enumerate(systems)]
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    atoms = [s.n_atoms for s in systems]
    out = {"workload": f"{n_mol} molecules of 3-60 atoms (log-uniform, seed 3000; species Si/A/B, each atom on its "
                       "species' grid: Si 60x306, A/B 80x434 points), batch sizes log-uniform in [20, 400]; one step "
                       "= H + n of every molecule; P = X X^T / 64 (rank 64)",
           "molecules": n_mol, "atoms": int(sum(atoms)), "points": int(sum(s.n_points for s in systems)),
           "generate_s": gen_s}

    def timed(fn, k=steps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    t0 = time.perf_counter()
    g = nao.Grid(systems, device=device, batch_points=bs, capture_graph=1, **BENCH_SPLIT_OPTS)
    torch.cuda.synchronize()
    out["create_s"] = time.perf_counter() - t0
    bo, _, ro, _ = g.batches()
    Pb, Nb = np.diff(bo), np.diff(ro)
    out["batches"] = {"count": int(len(Pb)), "points_min": int(Pb.min()), "points_max": int(Pb.max()),
                      "points_mean": float(Pb.mean()), "basis_min": int(Nb.min()), "basis_max": int(Nb.max()),
                      "basis_mean": float(Nb.mean()), "basis_pct": [int(x) for x in np.percentile(Nb, [5, 50, 95])]}
    Hs = [torch.empty((m["n_basis"], m["n_basis"]), dtype=torch.float64, device=dev) for m in g.systems]
    ns = [torch.empty(m["n_points"], dtype=torch.float64, device=dev) for m in g.systems]
    nes = [torch.empty(1, dtype=torch.float64, device=dev) for _ in g.systems]
    for prec in ("split", "fp64"):
        ms = timed(lambda: (g.integrate_h_many(vs, prec=prec, Hs=Hs, stream=stream),
                            g.update_density_many(Ps, prec=prec, ns=ns, nes=nes, stream=stream)),
                   k=steps if prec == "split" else 1)
        out[f"grouped_{prec}_ms_per_step"] = ms
        out[f"grouped_{prec}_points_per_s"] = out["points"] / (ms / 1e3)
    tw, tuned = nao.nao_get_tuning(g.h)
    out["tuning"] = {"buckets_timed": int(tuned), "tile_widths": sorted(set(int(x) for x in tw[Nb > 0]))}
    out["gflops_algorithmic_split"] = (g.info.flops_h + g.info.flops_n) / (out["grouped_split_ms_per_step"] / 1e3) / 1e9
    out["speedup_split_vs_fp64"] = out["grouped_fp64_ms_per_step"] / out["grouped_split_ms_per_step"]
    g.sync()
    g.close()
    if n_mol <= per_molecule_max:
        # one handle per molecule with the library's default options, one alive at a time (each
        # takes its own evaluation chunks, and a hundred of them at once would not fit the
        # device): the per-molecule step is the sum of every molecule's own timed step
        ms_s = 0.0
        for k, (sk, b) in enumerate(zip(systems, bs)):
            h = nao.Grid(sk, device=device, max_batch_points=b, **BENCH_SPLIT_OPTS)
            ms_s += timed(lambda: (h.integrate_h(vs[k], prec="split", H=Hs[k], stream=stream),
                                   h.update_density(Ps[k], prec="split", n=ns[k], ne=nes[k], stream=stream)))
            h.sync()
            h.close()
        out.update({"per_molecule_split_ms_per_step": ms_s,
                    "speedup_grouped": ms_s / out["grouped_split_ms_per_step"]})
    return out


def periodic(device: int, n_grid: int = 48, n_k: int = 4, steps: int = 3) -> dict:
    """Periodic silicon: the conventional diamond cell (10.26 bohr, 8 atoms, the diamond64 basis),
    its periodic images as the atoms of a finite system on the cell's points. h^uc and s^uc on the
    split path, then h(k) and s(k) by the Bloch sum on an n_k^3 k mesh."""
    import numpy as np
    import torch

    from paper_1912_06636_gb300 import nao, synth

    a = 10.26
    base = [[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]
    frac = base + [[x + 0.25 for x in f] for f in base]
    lat = np.eye(3) * a
    s = synth.periodic_cell(lat, frac, [0] * 8, [synth.silicon_species(1)], n_grid=n_grid, max_batch_points=300)
    xyz, atom, cell = nao.nao_periodic_images(s.atom_xyz, lat, float(np.max(s.fn_cutoff)))
    simg = synth.image_system(s, xyz, atom)
    fm, fi = nao.nao_periodic_basis_map(s, atom)
    u = (np.arange(n_k) + 0.5) / n_k - 0.5
    kf = np.stack(np.meshgrid(u, u, u, indexing="ij"), -1).reshape(-1, 3)
    dev = torch.device("cuda", device)
    kpts = torch.from_numpy(kf @ (2 * np.pi * np.linalg.inv(lat).T)).to(dev)
    fm_d, fi_d = torch.from_numpy(fm).to(dev), torch.from_numpy(fi).to(dev)
    cell_d = torch.from_numpy(np.ascontiguousarray(cell, dtype=np.int32)).to(dev)
    v = torch.from_numpy(synth.periodic_potential(s)).to(dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"periodic Si, conventional diamond cell 10.26 bohr, 8 atoms x 25 basis functions, "
                       f"{len(atom)} images (N_rs = {len(fm)}), {n_grid}^3 = {s.n_points} cell points "
                       f"(periodic trapezoid rule), batches <= 300 points, {n_k}^3 = {len(kf)} k points; "
                       "h^uc and s^uc split (11 slices)"}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    with nao.Grid(simg, device=device, max_batch_points=300, split_slices=11) as g:
        H = torch.empty((g.nb, g.nb), dtype=torch.float64, device=dev)
        S = torch.empty((g.nb, g.nb), dtype=torch.float64, device=dev)
        hk = torch.empty((len(kf), s.n_basis, s.n_basis, 2), dtype=torch.float64, device=dev)
        ms_h = timed(lambda: g.integrate_h(v, prec="split", H=H, stream=stream))
        ms_s = timed(lambda: g.overlap(prec="split", S=S, stream=stream))
        ms_k = timed(lambda: nao.nao_bloch_sum(H, fm_d, fi_d, cell_d, lat, kpts, s.n_basis, stream=stream, out=hk))
        g.sync()
    out.update({"h_uc_ms": ms_h, "h_uc_points_per_s": s.n_points / (ms_h / 1e3), "s_uc_ms": ms_s,
                "bloch_sum_ms": ms_k, "k_points_per_s": len(kf) / (ms_k / 1e3)})
    return out


def h_tile_area(n_basis, k_cols, tile_width, tile_rows: int = 128):
    """Issued and useful MMA area (rows x columns x K) of the split H contraction: per batch, the
    tile_rows x tile_width tiles that reach the upper triangle (i <= j) of its N x N block, against
    the triangle's own N (N + 1) / 2 elements (the part FLOP_H counts), both times the batch's K."""
    issued = useful = 0
    for n, k, tn in zip(n_basis, k_cols, tile_width):
        n, k, tn = int(n), int(k), int(tn)
        if n <= 0 or tn <= 0:
            continue
        useful += k * n * (n + 1) // 2
        for i0 in range(0, n, tile_rows):
            j_first = (i0 // tn) * tn  # the first column tile that reaches i0 <= j
            issued += k * tile_rows * tn * len(range(j_first, n, tn))
    return issued, useful


def g_split_pairs(g) -> int:
    """Slice products per contraction on the split path: S (S + 1) / 2 for S slices."""
    S = int(g.split_slices)
    return S * (S + 1) // 2


# ---------------------------------------------------------------------------------------
def workload_name(args) -> str:
    if args.config == 0:
        return "water3: 3-atom molecule, 20 basis functions, 40x110 points per atom = 13,200 points, batches <= 200"
    if args.config == 1 and args.cells != 2:
        return (f"diamond{8 * args.cells ** 3}: {8 * args.cells ** 3}-atom diamond-lattice cluster, 25 basis functions "
                "per atom, 60x306 points per atom, batches <= 300 points (profiling case)")
    if args.config == 2 and args.slab_layers != 15:
        return (f"slab{25 * args.slab_layers}: {args.slab_layers} layers of the slab (5x5 per layer), 40 basis functions "
                "per atom, 80x434 points per atom, batches <= 200 points (profiling case)")
    return WORKLOADS[args.config]


def bench_digits(args) -> str:
    return args.digits if args.digits is not None else BENCH_DIGITS.get(args.config, "bf16")


def bench_slices(args) -> int:
    if args.slices is not None:
        return args.slices
    if bench_digits(args) == "e4m3":
        return BENCH_SLICES_E4M3.get(args.config, 14)
    return BENCH_SLICES.get(args.config, 12)


def make_workload(config: int, device: str, cells: int = 2, layers: int = 15):
    from paper_1912_06636_gb300 import synth

    kw = {1: {"cells": cells}, 2: {"layers": layers}}.get(config, {})
    s = synth.config(config, **kw)
    v = s.potential()
    # the slab's P is X X^T / 64 with X nb x 64 (a dense 15000 x 15000 product would dominate the set-up)
    P = synth.density_matrix(s, config, rank=64 if config == 2 else None)
    return s, v, P


def _sample(s, n, seed):
    import numpy as np

    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(s.n_points, size=min(int(n), s.n_points), replace=False))


def _oracle_rate(s, v, P, idx):
    """Single-thread oracle on the points idx: (points/s, seconds of H, seconds of n)."""
    import oracle

    o = oracle.Oracle(s)
    t0 = time.perf_counter()
    o.hamiltonian(s.pt_xyz[idx], s.pt_w[idx], v[idx])
    t1 = time.perf_counter()
    o.density(s.pt_xyz[idx], P, s.pt_w[idx])
    t2 = time.perf_counter()
    return len(idx) / (t2 - t0), t1 - t0, t2 - t1


def calibrate_sample(s, v, P, seconds: float, seed: int = 12344) -> int:
    """Points of a sample that the single-thread oracle finishes in about `seconds` (from a
    2,000-point trial run)."""
    rate, _, _ = _oracle_rate(s, v, P, _sample(s, 2000, seed))
    return int(max(1000, min(s.n_points, rate * seconds)))


def cpu_baseline(s, v, P, n_sample: int, seed: int = 12345):
    """The FP64 oracle as it stands, on a seeded sample of the workload's points (1 thread)."""
    idx = _sample(s, n_sample, seed)
    rate, th, tn = _oracle_rate(s, v, P, idx)
    return {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(idx)} seeded points of the workload (H over those points, then n on them): "
                      f"H {th:.1f} s + n {tn:.1f} s"}


def _oracle_chunk(job):
    """One worker's share of the all-cores oracle baseline: H over its points, then n on them."""
    sub, v, P = job
    import oracle

    o = oracle.Oracle(sub)
    t0 = time.perf_counter()
    o.hamiltonian(sub.pt_xyz, sub.pt_w, v)
    o.density(sub.pt_xyz, P, sub.pt_w)
    return time.perf_counter() - t0


def _oracle_pool(procs: int):
    import concurrent.futures
    import multiprocessing

    return concurrent.futures.ProcessPoolExecutor(procs, mp_context=multiprocessing.get_context("spawn"))


def cpu_baseline_all_cores(s, v, P, n_sample: int, seed: int = 12345, ex=None):
    """The same oracle in one process per host core (spawned: this process has used the GPU), each on
    a slice of a seeded sample; wall time of the parallel part (the pool and its imports are
    started before the clock)."""
    import dataclasses

    import numpy as np

    procs = os.cpu_count() or 1
    idx = _sample(s, n_sample, seed)
    parts = np.array_split(idx, procs)
    jobs = [(dataclasses.replace(s, pt_xyz=s.pt_xyz[p], pt_w=s.pt_w[p]), v[p], P) for p in parts]
    own = ex is None
    if own:
        ex = _oracle_pool(procs)
    try:
        list(ex.map(_oracle_chunk, [(dataclasses.replace(s, pt_xyz=s.pt_xyz[:8], pt_w=s.pt_w[:8]), v[:8], P)] * procs))
        t0 = time.perf_counter()
        busy = list(ex.map(_oracle_chunk, jobs))
        wall = time.perf_counter() - t0
    finally:
        if own:
            ex.shutdown()
    return {"value": len(idx) / wall, "unit": "points/s", "cores": procs, "kind": "oracle",
            "sample": f"{len(idx)} seeded points in {procs} processes (H then n each); wall {wall:.1f} s, "
                      f"busiest process {max(busy):.1f} s"}


def run_reference(args):
    """The oracle as it stands, on every host core (one process per core), on seeded samples of
    the workload: each step is one sample (H then n), sized from a single-thread trial so that
    a step takes about --cpu-seconds / 3 of wall time on all cores."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    s, v, P = make_workload(args.config, "cpu", args.cells, args.slab_layers)
    procs = os.cpu_count() or 1
    n_sample = max(200 * procs, calibrate_sample(s, v, P, procs * args.cpu_seconds / 3.0))
    times = []
    with _oracle_pool(procs) as ex:
        for k in range(args.warmup + args.steps):
            times.append(cpu_baseline_all_cores(s, v, P, n_sample, seed=12345 + k, ex=ex))
    timed = times[args.warmup:]
    val = statistics.mean(t["value"] for t in timed)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s.n_points / val,
            "ms_per_step_kind": (f"extrapolated: the whole grid ({s.n_points} points) at the rate measured on "
                                 f"{n_sample}-point samples (each step times one sample)"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "points/s", "cores": procs, "kind": "oracle",
                             "sample": timed[0]["sample"] + " per step"},
            "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import __graft_entry__

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    __graft_entry__.build()
    from paper_1912_06636_gb300 import nao, replicas

    prec = args.prec or "split"
    s, v_np, P_np = make_workload(args.config, f"cuda:{local_rank}", args.cells, args.slab_layers)
    dev = torch.device("cuda", local_rank)
    t0 = time.perf_counter()
    slices, digits = bench_slices(args), bench_digits(args)
    extra = {"scratch_bytes": args.scratch_mb << 20} if args.scratch_mb > 0 else {}
    extra["split_digits"] = 1 if digits == "e4m3" else 0
    g = nao.Grid(s, device=local_rank, max_batch_points=s.max_batch_points, split_slices=slices, **extra)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    info = g.info
    v = torch.from_numpy(v_np).to(dev)
    P = torch.from_numpy(P_np).to(dev)
    H = torch.empty((g.nb, g.nb), dtype=torch.float64, device=dev)
    n = torch.empty(g.n_points, dtype=torch.float64, device=dev)
    ne = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step(p=prec):
        g.integrate_h(v, prec=p, H=H, stream=stream)
        g.update_density(P, prec=p, n=n, ne=ne, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.sync()

    sampler = ClockSampler(local_rank)
    sampler.start()
    nao.nao_profile_enable(g.h, True)
    nao.nao_profile_read(g.h, reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed")  # profilers can select the timed steps by this range
    for k in range(args.steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    prof = nao.nao_profile_read(g.h, reset=True)
    nao.nao_profile_enable(g.h, False)
    g.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][1])
    # all ranks' points over the slowest rank's time (replicas: no data-path collective)
    value, total_ms, _ = replicas.aggregate(args.steps * g.n_points, total_ms, dev)
    bo, _, ro, _ = g.batches()
    Pb, Nb = np.diff(bo), np.diff(ro)
    Ppad = (Pb + 15) // 16 * 16
    scratch_gb = float(np.sum(Nb * Ppad * 8 * 5)) / 1e9

    # roofline of the dominant kernel family (per launch: algorithmic work / event-timed duration)
    fam = max(prof, key=lambda k: prof[k][1])
    launches, fam_ms = prof[fam]
    pairs = {"split": g_split_pairs(g)}.get(prec, 1)
    work = {"h_fp64": info.flops_h, "h_fp32": info.flops_h, "h_split": pairs * info.flops_h,
            "n_fp64": info.flops_n, "n_fp32": info.flops_n, "n_split": pairs * info.flops_n}
    roofline = None
    if fam in work and fam_ms > 0:
        achieved = work[fam] * args.steps / (fam_ms / 1e3) / 1e12
        if fam.endswith("fp64") or fam.endswith("fp32"):
            peak, peak_src = alu_peak(fam[-4:])
            roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": None, "kernel": fam, "peak_source": peak_src}
        else:
            mp = measured_peaks()
            pk, pk_s = mp.get("bf16_tflops", 1900.0), mp.get("bf16_tflops_sustained", 1700.0)
            src_pk = "MEASURED_PEAKS.json bf16_tflops (burst; of measured)" if "bf16_tflops" in mp else "fallback 1.9 PFLOP/s"
            if digits == "e4m3":  # e4m3 MMAs: the measured bf16 peak times the nominal fp8/bf16 ratio (4.5 / 2.25)
                pk, pk_s = 2.0 * pk, 2.0 * pk_s
                src_pk += " x 2 (nominal fp8 / bf16 dense ratio: the e4m3 peak)"
            roofline = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                        "traffic": None, "kernel": fam,
                        "work": f"{pairs} slice products x algorithmic FLOPs (sum_b 4 P_b N_b (N_b+1) for H)",
                        "peak_source": src_pk, "frac_of_sustained": achieved / pk_s}
        roofline.update({"launches": launches, "avg_launch_ms": fam_ms / max(launches, 1)})
        tk = (args.config, fam, int(g.split_slices) if prec == "split" else 0)
        if tk in TRAFFIC_PER_FLOP_H and launches:
            per_flop, src = TRAFFIC_PER_FLOP_H[tk]
            roofline["traffic"] = per_flop * info.flops_h * args.steps / launches
            roofline["traffic_unit"] = "bytes per launch"
            roofline["traffic_source"] = src + " (bytes per FLOP_H x this run's FLOP_H per launch)"
    gpu_launches = int(sum(l for l, _ in prof.values()))
    tuning = None
    if prec == "split":
        tw, timed = nao.nao_get_tuning(g.h)
        tuning = {"buckets_timed": timed, "batches_tile48": int(np.sum(tw == 48)), "batches_tile32": int(np.sum(tw == 32))}
        if roofline is not None and fam == "h_split":
            try:  # the share of the issued MMA area that is the work FLOP_H counts
                issued, useful = h_tile_area(Nb, 4 * Ppad, tw)
                roofline["useful_area_frac"] = useful / issued
                roofline["issued_tflops"] = roofline["achieved"] * issued / useful
            except Exception as e:  # reported, never fatal
                roofline["useful_area_frac"] = f"unavailable: {type(e).__name__}: {e}"
            if tk in TRAFFIC_PER_ISSUED_FLOP and isinstance(roofline.get("issued_tflops"), float) and digits == "e4m3":
                per_flop, src = TRAFFIC_PER_ISSUED_FLOP[tk]
                issued_per_launch = roofline["issued_tflops"] * 1e12 * roofline["avg_launch_ms"] / 1e3
                roofline["traffic"] = per_flop * issued_per_launch
                roofline["traffic_unit"] = "bytes per launch"
                roofline["traffic_source"] = (src + " (DRAM bytes per issued tensor FLOP of one 125-atom slab launch "
                                              "x this run's issued FLOP per launch)")

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "split": f"{digits}x-slices+f64"}[prec],
        "data": "synthetic",
        "config": {"workload": workload_name(args), "precision": prec, "parallelism": f"replicas{world}",
                   "split_slices": slices if prec == "split" else None,
                   "split_digits": digits if prec == "split" else None,
                   "l2": f"inputs/working set larger than L2: {scratch_gb:.1f} GB of evaluated basis functions "
                         "written and re-read per step",
                   "n_points": g.n_points, "n_basis": g.nb, "n_batches": int(info.n_batches),
                   "max_batch_basis": int(info.max_batch_basis)},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "gflops_algorithmic": (info.flops_h + info.flops_n) / (total_ms / args.steps / 1e3) / 1e9,
        "create_s": create_s,
        "roofline": roofline, "gpu_launches": gpu_launches, "clocks": clocks, "tuning": tuning,
        "kernel_ms_per_step": {k: ms / args.steps for k, (l, ms) in prof.items() if l},
    }

    if not args.no_e2e:
        Hh = torch.empty((g.nb, g.nb), dtype=torch.float64).pin_memory().numpy()
        nh = torch.empty(g.n_points, dtype=torch.float64).pin_memory().numpy()
        vh = torch.from_numpy(v_np).pin_memory().numpy()
        Ph = torch.from_numpy(P_np).pin_memory().numpy()
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            nao.nao_integrate_h_host(g.h, vh, 3, prec, Hh, stream)
            nao.nao_update_density_host(g.h, Ph, prec, nh, stream)
        dt = (time.perf_counter() - t0) / e2e_steps
        line["e2e"] = {"value": g.n_points / dt, "unit": "points/s",
                       "h2d_bytes_per_step": int(8 * (g.n_points + g.nb * g.nb)),
                       "d2h_bytes_per_step": int(8 * (g.nb * g.nb + g.n_points + 1))}

    if not args.no_compare:
        other = {}
        for p in ("fp64", "fp32", "split"):
            if p == prec:
                continue
            try:
                step(p)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step(p)
                b.record(stream)
                torch.cuda.synchronize()
                other[p] = {"points_per_s": g.n_points / (a.elapsed_time(b) / 1e3), "ms_per_step": a.elapsed_time(b)}
                if p == "fp64":
                    line["fp64_points_per_s"] = other[p]["points_per_s"]
                    line["speedup_vs_fp64"] = value / other[p]["points_per_s"]
            except nao.NaoError as e:
                other[p] = {"unavailable": str(e)}
        # the split path with the other digit format, at the slice count its parity tests check
        od = "e4m3" if digits == "bf16" else "bf16"
        os_ = BENCH_SLICES_E4M3.get(args.config, 14) if od == "e4m3" else BENCH_SLICES.get(args.config, 11)
        try:
            g3 = nao.Grid(s, device=local_rank, max_batch_points=s.max_batch_points, split_slices=os_,
                          split_digits=1 if od == "e4m3" else 0)
            for rep in range(2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g3.integrate_h(v, prec="split", H=H, stream=stream)
                g3.update_density(P, prec="split", n=n, ne=ne, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
            g3.sync()
            other[f"split_{od}_{os_}_slices"] = {"points_per_s": g.n_points / (a.elapsed_time(b) / 1e3),
                                                  "ms_per_step": a.elapsed_time(b)}
            g3.close()
        except nao.NaoError as e:
            other[f"split_{od}_{os_}_slices"] = {"unavailable": str(e)}
        # the split path at the library's default slice count
        d = nao.nao_default_options().split_slices
        if d != slices or digits != "bf16":
            try:
                g2 = nao.Grid(s, device=local_rank, max_batch_points=s.max_batch_points)
                g2.integrate_h(v, prec="split", H=H, stream=stream)
                g2.update_density(P, prec="split", n=n, ne=ne, stream=stream)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g2.integrate_h(v, prec="split", H=H, stream=stream)
                g2.update_density(P, prec="split", n=n, ne=ne, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                g2.sync()
                other[f"split_{d}_slices"] = {"points_per_s": g.n_points / (a.elapsed_time(b) / 1e3),
                                              "ms_per_step": a.elapsed_time(b)}
                g2.close()
            except nao.NaoError as e:
                other[f"split_{d}_slices"] = {"unavailable": str(e)}
        line["other_precisions"] = other
        # the extensions on the same workload, one untimed and one timed call each: the density
        # gradient (split, FP64) and Hessian (FP64, FP32, split), H with the meta-GGA term (split), the
        # local Pulay matrix elements (FP64, FP32)
        deriv = {}
        gbuf = torch.empty((3, g.n_points), dtype=torch.float64, device=dev)
        hbuf = torch.empty((6, g.n_points), dtype=torch.float64, device=dev)
        vtau = torch.full((g.n_points,), 0.25, dtype=torch.float64, device=dev)
        mbuf = torch.empty((3, g.nb, g.nb), dtype=torch.float64, device=dev)
        sbuf = torch.empty((3, g.nb, g.nb), dtype=torch.float64, device=dev)
        calls = {
            "gradient_split": lambda: g.density_gradient(P, prec="split", n=n, grad=gbuf, ne=ne, stream=stream),
            "gradient_fp64": lambda: g.density_gradient(P, prec="fp64", n=n, grad=gbuf, ne=ne, stream=stream),
            "hessian_fp64": lambda: g.density_hessian(P, prec="fp64", n=n, grad=gbuf, hess=hbuf, ne=ne, stream=stream),
            "hessian_fp32": lambda: g.density_hessian(P, prec="fp32", n=n, grad=gbuf, hess=hbuf, ne=ne, stream=stream),
            "hessian_split": lambda: g.density_hessian(P, prec="split", n=n, grad=gbuf, hess=hbuf, ne=ne, stream=stream),
            "h_with_tau_split": lambda: g.integrate_h_tau(v, vtau, prec="split", H=H, stream=stream),
            "pulay_matrices_fp64": lambda: g.pulay_matrices(v, prec="fp64", M=mbuf, S=sbuf, stream=stream),
            "pulay_matrices_fp32": lambda: g.pulay_matrices(v, prec="fp32", M=mbuf, S=sbuf, stream=stream),
        }
        for name, call in calls.items():
            try:
                call()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                torch.cuda.synchronize()
                g.sync()
                deriv[name] = {"ms": a.elapsed_time(b), "points_per_s": g.n_points / (a.elapsed_time(b) / 1e3)}
            except nao.NaoError as e:
                deriv[name] = {"unavailable": str(e)}
        line["extensions"] = deriv

    if rank == 0 and world == 1 and not args.no_serve and args.serve_requests > 0:
        g.close()
        line["serving"] = serving(args.serve_requests, local_rank, args.serve_fp64_requests)
    if rank == 0 and world == 1 and args.grouped_molecules > 0:
        if g.h:
            g.close()
        line["grouped"] = grouped(args.grouped_molecules, local_rank)

    if rank == 0 and world == 1 and not args.no_periodic:
        if g.h:
            g.close()
        try:
            line["periodic"] = periodic(local_rank)
        except nao.NaoError as e:
            line["periodic"] = {"unavailable": str(e)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n1 = calibrate_sample(s, v_np, P_np, args.cpu_seconds)
        line["cpu_baseline"] = cpu_baseline(s, v_np, P_np, n1)
        try:
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(s, v_np, P_np, (os.cpu_count() or 1) * n1)
        except Exception as e:  # the single-thread figure stands on its own
            line["cpu_baseline"]["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    if g.h:
        g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
