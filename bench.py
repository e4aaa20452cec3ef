#!/usr/bin/env python
"""Benchmark of the multiscale fit on one GB300 (or N, one process per GPU).

One step = one pass of the whole hot path over the synthetic workload, with the
inputs already resident in HBM:
  ms_build_hierarchy_dev  (level grids, cell binning, CSR of A_l and B_kj)
  ms_fit_dev              (preconditioner rows by the trained network, then Jacobi
                           sweeps on T' + per-level CG on D in one persistent kernel)
  ms_evaluate_dev         (approximant at a 256^2 query grid)
Workload: d=2, 8 levels of scrambled Halton points, N_j = 64*4^(j-1) (1,398,080 points),
h_j = N_j^-1/2, delta_j = 4 h_j, Wendland phi_{2,1}, f = 20 Gaussians + 0.1 sin(8 pi x) sin(8 pi y).
The timed path is learned-PCG MIXED (FP32 mat-vecs, FP64 dots and refinement, FSAI rows
predicted by the network trained beforehand on levels 1-4, training timed separately);
plain FP64 CG+Jacobi and the other variants are timed beside it.
`--impl reference` times the CPU FP64 oracle instead.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fit time at rel-err 1e-8: learned-PCG FP32 vs plain FP64 (ms); mat-vec GB/s"
REL_TOL = 1e-10


def halton_points(levels):
    """Points of the Halton hierarchy with N_j = 64 * 4^(j-1), j = 1..levels."""
    return sum(64 * 4 ** j for j in range(levels))


def workload_label(levels):
    return (f"halton{levels}_d2_nu4_w21: d=2, {levels} levels scrambled Halton N_j=64*4^(j-1) "
            f"({halton_points(levels):,} points), delta_j=4*N_j^-1/2, Wendland phi_{{2,1}}, "
            "f=20 Gaussians+0.1 sin(8pi x)sin(8pi y)")



def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--levels", type=int, default=8)
    p.add_argument("--query-side", type=int, default=256)
    p.add_argument("--train-epochs", type=int, default=100)
    p.add_argument("--cpu-levels", type=int, default=6, help="levels of the oracle's bounded sample")
    p.add_argument("--ref-levels", type=int, default=5, help="levels per step of the reference arm")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-variants", action="store_true", help="skip the comparison paths")
    p.add_argument("--no-nu8", action="store_true", help="skip the nu=8, phi_{2,2} block")
    p.add_argument("--no-batch", action="store_true", help="skip the multi-RHS batching block")
    p.add_argument("--no-paper", action="store_true", help="skip the paper-grid (Section 5) block")
    p.add_argument("--cfg3", action="store_true", help="also run the 3-D configuration (about a minute)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def max_over_ranks(x, world_size, device):
    """The slowest rank's value: every rank fits its own replica of the workload (no data-path
    collective), so the job's step time is the maximum over the ranks."""
    if world_size <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mf_candidates(w):
    """Candidate pairs of the matrix-free mat-vec: for every point, the points of the 3^d cells (cell
    size delta_l, the level's bounding box as origin) around its own cell in its level."""
    import numpy as np
    total = 0
    for l, X in enumerate(w.levels):
        delta = w.nu * w.h[l]
        lo = X.min(axis=0)
        c = np.floor((X - lo) / delta).astype(np.int64)
        G = c.max(axis=0) + 1
        c = np.minimum(c, G - 1)
        key = c[:, 0] * G[1] + c[:, 1]
        cnt = np.bincount(key, minlength=int(G[0] * G[1])).reshape(G[0], G[1])
        pad = np.pad(cnt, 1)
        box = sum(pad[1 + dx:1 + dx + G[0], 1 + dy:1 + dy + G[1]] for dx in (-1, 0, 1) for dy in (-1, 0, 1))
        total += int(box[c[:, 0], c[:, 1]].sum())
    return total


def recorded_traffic(profile="k_fit_learned_halton8.md"):
    """DRAM traffic per launch of the solve kernel from the committed ncu summary, or None when
    the kernel's source has changed since the counters were taken (sha256 lines of the summary)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    traffic = None
    for line in text.splitlines():
        if line.startswith("kernel_source_sha256 "):
            name, digest = line[len("kernel_source_sha256 "):].split(":")
            path = os.path.join(ROOT, "paper_2503_04914_gb300", "csrc", name.strip())
            try:
                cur = hashlib.sha256(open(path, "rb").read()).hexdigest()
            except OSError:
                return None
            if cur != digest.strip():
                return None
        elif line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":")[1])
    return traffic


def cpu_baseline(levels, query_n, reps=1):
    """Time the CPU oracle (as it stands) on a bounded sample in a single-threaded subprocess."""
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import multiscale as om
from paper_2503_04914_gb300 import inputs
w = inputs.halton_hierarchy(L={levels})
Q = inputs.query_grid(256, 2)[:{query_n}]
ts = []
for _ in range({reps}):
    t = time.perf_counter()
    a, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, 2, 1)
    s = om.evaluate(w.levels, a, w.h, w.nu, 2, 1, Q)
    ts.append(time.perf_counter() - t)
print(json.dumps({{"N": w.N, "times": ts}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ reference arm (the oracle)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    reps = args.warmup + args.steps
    out = cpu_baseline(args.ref_levels, 1024, reps=reps)
    ts = out["times"][args.warmup:]
    n_work = halton_points(args.levels)
    scale = n_work / out["N"]
    ms_step = 1000.0 * statistics.mean(ts) * scale
    sample = (f"oracle fit_sequential + evaluate on the first {args.ref_levels} levels of the workload "
              f"({out['N']} points, 1024 queries), single-threaded, scaled by points ({n_work}/{out['N']})")
    line = {"impl": "reference", "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args.levels), "rel_tol": REL_TOL},
            "cpu_baseline": {"value": ms_step, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms_step, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2503_04914_gb300 import build as B
    from paper_2503_04914_gb300 import inputs, ms
    B.build()
    ms.load()

    w = inputs.halton_hierarchy(L=args.levels)
    pts = torch.from_numpy(w.points).cuda()
    f = torch.from_numpy(w.f).cuda()
    Qh = inputs.query_grid(args.query_side, 2)
    Q = torch.from_numpy(Qh).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    n = w.n_per_level

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # train the network once (levels 1-4 of this hierarchy), outside the timed region
    Ht = ms.Hierarchy(2, n, pts, w.h, precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED,
                      wendland_d=2, wendland_k=1, nu=w.nu)
    train = Ht.train_precond([0, 1, 2, 3], epochs=args.train_epochs)
    params = Ht.precond_params()
    Ht.close()
    params3 = None  # the 3-D network (the --cfg3 block trains it)
    Q3 = torch.from_numpy(inputs.query_grid(32, 3)).cuda()  # 32^3 queries for 3-D workloads

    def step(prec, precond=ms.MS_PRECOND_NONE, inter_tol=0.0, wl=None, pts_=None, f_=None, **extra):
        wl = wl or w
        pts_ = pts if pts_ is None else pts_
        f_ = f if f_ is None else f_
        opts = ms.ms_default_opts(wendland_d=wl.wendland_d, wendland_k=wl.wendland_k, nu=wl.nu, precision=prec,
                                  precond=precond, inter_tol=inter_tol, **extra)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        hnd = ms.ms_build_hierarchy(wl.d, wl.n_per_level, pts_, wl.h, opts)
        if precond == ms.MS_PRECOND_LEARNED:
            ms.ms_precond_params(hnd, wl.d, params if wl.d == 2 else params3)
        alpha, st = ms.ms_fit(hnd, f_, REL_TOL)
        e1.record(stream)
        s = ms.ms_evaluate(hnd, alpha, Q if wl.d == 2 else Q3)  # queries of the workload's dimension
        e2.record(stream)
        torch.cuda.synchronize()
        info = ms.ms_hierarchy_info(hnd)
        ms.ms_destroy(hnd)
        return {"total": e0.elapsed_time(e2), "eval": e1.elapsed_time(e2), "stats": st, "info": info,
                "alpha": alpha}

    def timed(k, *a, **kw):
        recs = []
        for _ in range(k):
            flush.fill_(1.0)  # L2 flush between steps (256 MB write), outside the timed events
            barrier()
            recs.append(step(*a, **kw))
            barrier()
        return recs

    def summary(recs):
        st = recs[-1]["stats"]
        return {"ms_per_step": statistics.mean(r["total"] for r in recs),
                "fit_ms": statistics.mean(r["stats"]["fit_ms"] for r in recs),
                "build_ms": statistics.mean(r["info"]["build_ms"] for r in recs),
                "cg_iterations": st["cg_iterations"], "rel_residual_max": max(st["rel_residual"]),
                "precond_fallbacks": st["precond_fallbacks"],
                "phase_ms": {k: round(v, 3) for k, v in st["phase_ms"].items()}}

    HEAD = (ms.MS_PREC_MIXED, ms.MS_PRECOND_LEARNED)
    for _ in range(args.warmup):
        step(*HEAD)
    clocks = ClockSampler(local)
    lc0 = ms.ms_launch_count()
    clocks.start()
    t_wall = time.perf_counter()
    recs = timed(args.steps, *HEAD)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    launches = (ms.ms_launch_count() - lc0) / args.steps
    ms_step = max_over_ranks(statistics.mean(r["total"] for r in recs), ws, "cuda")
    last = recs[-1]
    st, info = last["stats"], last["info"]

    out = {}
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm = float(peaks["hbm_gbs"])
        fit_ms = statistics.mean(r["stats"]["fit_ms"] for r in recs)
        fit_bytes = st["matvec_bytes"]
        achieved = fit_bytes / (fit_ms * 1e-3) / 1e9
        out["roofline"] = {"kernel": "k_fit<MIXED> (persistent Jacobi / learned-PCG solve)", "bound": "hbm",
                           "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                           "peak_kind": f"{peak_kind} hbm_gbs",
                           "traffic": recorded_traffic() if args.levels == 8 and args.train_epochs == 100 else None,
                           "traffic_source": "profiles/k_fit_learned_halton8.md (1-pass ncu capture of this workload)",
                           "algorithmic_bytes_per_launch": fit_bytes, "launch_ms": fit_ms}
        out["learned_pcg"] = summary(recs)
        out["phases_ms"] = {"build": out["learned_pcg"]["build_ms"], "fit_incl_precond": None,
                            "fit_kernel": fit_ms, "evaluate": statistics.mean(r["eval"] for r in recs)}
        out["phases_ms"]["fit_incl_precond"] = (out["learned_pcg"]["ms_per_step"] - out["phases_ms"]["build"]
                                                - out["phases_ms"]["evaluate"])
        out["train"] = {"levels": [1, 2, 3, 4], "epochs": args.train_epochs, "extra_patches_per_point": 4, **train}
        out["nnz"] = {"A": info["nnz_A"], "B": info["nnz_B"]}

        if not args.no_variants:
            k2 = max(2, args.steps // 2)
            out["plain_fp64"] = summary(timed(k2, ms.MS_PREC_FP64))
            out["mixed_no_precond"] = summary(timed(k2, ms.MS_PREC_MIXED))
            out["mixed_exact_fsai"] = summary(timed(k2, ms.MS_PREC_MIXED, ms.MS_PRECOND_EXACT))
            out["algorithm2_schedule_fp64"] = summary(timed(1, ms.MS_PREC_FP64, inter_tol=REL_TOL))
            # the other CTAs-per-SM choice of the persistent solve kernel (autotuning evidence)
            out["learned_pcg_1cta_per_sm"] = summary(timed(k2, *HEAD, solve_ctas_per_sm=1))
            out["plain_fp64_1cta_per_sm"] = summary(timed(k2, ms.MS_PREC_FP64, solve_ctas_per_sm=1))
            # lanes per row chosen by timing (ms_opts.autotune); the first handle times, the rest hit the cache
            timed(1, *HEAD, autotune=1)
            rt = timed(k2, *HEAD, autotune=1)
            out["learned_pcg_autotuned"] = summary(rt)
            out["learned_pcg_autotuned"]["tpr_A"] = rt[-1]["info"]["tpr_A"]
            out["learned_pcg_autotuned"]["tpr_A_rule"] = info["tpr_A"]
            out["speedup_learned_vs_plain_fp64"] = out["plain_fp64"]["ms_per_step"] / ms_step
            # agreement of the headline coefficients with the plain FP64 fit (same hierarchy, same f)
            a0 = timed(1, ms.MS_PREC_FP64)[0]["alpha"]
            a1 = last["alpha"]
            out["rel_diff_vs_fp64_coefficients"] = float(torch.linalg.norm(a1 - a0) / torch.linalg.norm(a0))

        # stand-alone mat-vecs (sorted order): GB/s of the CSR kernels, matrix-free timing
        peaks_alu = {"fp32": ms.ms_peak_probe(ms.MS_PROBE_FP32), "fp64": ms.ms_peak_probe(ms.MS_PROBE_FP64),
                     "xu": ms.ms_peak_probe(ms.MS_PROBE_XU)}
        H = ms.Hierarchy(2, n, pts, w.h, precision=ms.MS_PREC_MIXED, wendland_d=2, wendland_k=1, nu=w.nu)
        N = w.N
        x = torch.randn(N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        mv = {}
        for name, op, nnz, vb in [("A64", ms.MS_APPLY_A64, info["nnz_A"], 8), ("A32", ms.MS_APPLY_A32, info["nnz_A"], 4),
                                  ("AMF32", ms.MS_APPLY_AMF32, info["nnz_A"], 0), ("B64", ms.MS_APPLY_B64, info["nnz_B"], 8)]:
            for _ in range(3):
                H.apply(op, x, y, sorted_order=True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            reps = 20
            ev[0].record(stream)
            for _ in range(reps):
                H.apply(op, x, y, sorted_order=True)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_ms = ev[0].elapsed_time(ev[1]) / reps
            if vb:
                # matrix (col + val) + row offsets + y write + one read of x (FP32 ops also convert x)
                b = nnz * (4 + vb) + N * (8 + 8 + 8) + (N * 12 if vb == 4 else 0)
                mv[name] = {"ms": t_ms, "GBps": b / (t_ms * 1e-3) / 1e9, "frac_hbm": b / (t_ms * 1e-3) / 1e9 / hbm,
                            "algorithmic_bytes": b}
            else:
                # matrix-free: bound by FP32 and XU issue; every candidate pair (points of the
                # 3^d cells around each point's cell) costs 13 FP32-pipe instructions and one
                # reciprocal square root (ms_matfree.cuh, d = 2, phi_{d,1})
                cand = mf_candidates(w)
                f32 = 13.0 * cand / (t_ms * 1e-3)
                xu = cand / (t_ms * 1e-3)
                mv[name] = {"ms": t_ms, "stored_entries_per_s": nnz / (t_ms * 1e-3), "candidate_pairs": cand,
                            "fp32_instr_per_s": f32, "frac_fp32": f32 / peaks_alu["fp32"],
                            "xu_per_s": xu, "frac_xu": xu / peaks_alu["xu"]}
        out["matvec"] = mv
        out["alu_peaks_measured"] = {"fp32_instr_per_s": peaks_alu["fp32"], "fp64_instr_per_s": peaks_alu["fp64"],
                                     "xu_per_s": peaks_alu["xu"], "probe": "ms_peak_probe (own FMA / rsqrt chains)"}
        H.close()

        # nu = 8, phi_{2,2} (ill-conditioned levels): learned-PCG MIXED vs plain FP64, one step each
        if not args.no_nu8:
            w8 = inputs.halton_hierarchy(L=args.levels, nu=8.0, wendland=(2, 2))
            p8, f8 = torch.from_numpy(w8.points).cuda(), torch.from_numpy(w8.f).cuda()
            H8 = ms.Hierarchy(2, w8.n_per_level, p8, w8.h, precision=ms.MS_PREC_MIXED,
                              precond=ms.MS_PRECOND_LEARNED, wendland_d=2, wendland_k=2, nu=8.0)
            train8 = H8.train_precond([0, 1, 2, 3], epochs=args.train_epochs)
            params8 = H8.precond_params()
            H8.close()
            saved = params
            params = params8
            r8 = timed(1, ms.MS_PREC_MIXED, ms.MS_PRECOND_LEARNED, wl=w8, pts_=p8, f_=f8)
            params = saved
            r8f = timed(1, ms.MS_PREC_FP64, wl=w8, pts_=p8, f_=f8)
            out["nu8_w22"] = {"workload": "as above with delta_j = 8 h_j and Wendland phi_{2,2}",
                              "learned_pcg": summary(r8), "plain_fp64": summary(r8f),
                              "train": {"levels": [1, 2, 3, 4], **train8},
                              "speedup": summary(r8f)["ms_per_step"] / summary(r8)["ms_per_step"]}
            del p8, f8

        # batching: 256 right-hand sides on one 6-level hierarchy (87,360 points), MIXED without
        # preconditioner, solved 32 per launch; against single-RHS fits of the first 16 of them
        if not args.no_batch:
            wb = inputs.halton_hierarchy(L=6)
            pb = torch.from_numpy(wb.points).cuda()
            Fb = np.stack([inputs.GaussianMixture(5, 2, 7000 + r)(wb.points) for r in range(256)], axis=1)
            Fb = torch.from_numpy(np.ascontiguousarray(Fb)).cuda()
            Hb = ms.Hierarchy(2, wb.n_per_level, pb, wb.h, precision=ms.MS_PREC_MIXED, wendland_d=2,
                              wendland_k=1, nu=wb.nu)
            Hb.fit(Fb[:, :32].contiguous(), REL_TOL)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev[0].record(stream)
            Ab, stb = Hb.fit(Fb, REL_TOL)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_batch = ev[0].elapsed_time(ev[1])
            t_single = []
            for r in range(16):
                fr = Fb[:, r].contiguous()
                flush.fill_(1.0)
                torch.cuda.synchronize()
                ev[0].record(stream)
                a1, _ = Hb.fit(fr, REL_TOL)
                ev[1].record(stream)
                torch.cuda.synchronize()
                t_single.append(ev[0].elapsed_time(ev[1]))
            agree = float(torch.linalg.norm(Ab[:, 15] - a1) / torch.linalg.norm(a1))
            Hb.close()
            out["batch_rhs"] = {"workload": "d=2, 6 Halton levels N_j=64*4^(j-1) (87,360 points), delta_j=4h_j, "
                                            "phi_{2,1}, 256 right-hand sides (seeded 5-Gaussian mixtures), MIXED",
                                "rhs": 256, "rhs_per_launch": 32, "batched_ms": t_batch,
                                "batched_ms_per_rhs": t_batch / 256, "single_ms_per_rhs": statistics.mean(t_single),
                                "speedup_per_rhs": statistics.mean(t_single) / (t_batch / 256),
                                "kernel_ms": stb["fit_ms"], "rel_residual_max": max(stb["rel_residual"]),
                                "rel_diff_column15_vs_single": agree}
            del pb, Fb, Ab

            # 64 independent hierarchies (3-7 levels, finest 4k-260k points) in one launch vs one by one
            wsb = inputs.batch_hierarchies()
            Hs = [ms.Hierarchy(2, wi.n_per_level, torch.from_numpy(wi.points).cuda(), wi.h,
                               precision=ms.MS_PREC_MIXED, wendland_d=2, wendland_k=1, nu=wi.nu) for wi in wsb]
            fsb = [torch.from_numpy(wi.f).cuda() for wi in wsb]
            handles = [Hi.handle for Hi in Hs]
            ms.ms_fit_batch(handles, fsb, REL_TOL)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev[0].record(stream)
            Ab, stb = ms.ms_fit_batch(handles, fsb, REL_TOL)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_b = ev[0].elapsed_time(ev[1])
            t_one = 0.0
            worst = 0.0
            for Hi, fi, ai in zip(Hs, fsb, Ab):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                ev[0].record(stream)
                a1, _ = Hi.fit(fi, REL_TOL)
                ev[1].record(stream)
                torch.cuda.synchronize()
                t_one += ev[0].elapsed_time(ev[1])
                worst = max(worst, float(torch.linalg.norm(ai - a1) / torch.linalg.norm(a1)))
            # the same batch as a prepared plan replayed from a CUDA graph (host work done once)
            plan = ms.BatchPlan(handles, fsb, REL_TOL)
            plan.launch(use_graph=True)
            plan.stats()
            t_graph = []
            for _ in range(3):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                ev[0].record(stream)
                plan.launch(use_graph=True)
                ev[1].record(stream)
                torch.cuda.synchronize()
                t_graph.append(ev[0].elapsed_time(ev[1]))
            stg = plan.stats()
            graph_diff = max(float(torch.linalg.norm(ag - ai) / torch.linalg.norm(ai)) for ag, ai in zip(plan.alphas, Ab))
            plan.close()
            out["batch_hierarchies"] = {
                "workload": "64 d=2 Halton hierarchies, L ~ U{3..7}, finest N log-uniform in [4096, 262144], "
                            "delta_j=4h_j, phi_{2,1}, one Gaussian-mixture RHS each, MIXED",
                "points": int(sum(wi.N for wi in wsb)), "batched_ms": t_b, "kernel_ms": stb[0]["fit_ms"],
                "one_by_one_ms": t_one, "speedup": t_one / t_b,
                "rel_residual_max": max(max(s["rel_residual"]) for s in stb),
                "rel_diff_vs_single_max": worst,
                "graph_replay_ms": statistics.mean(t_graph), "graph_rel_diff_vs_batched_max": graph_diff,
                "graph_rel_residual_max": max(max(s["rel_residual"]) for s in stg)}
            for Hi in Hs:
                Hi.close()
            # the same 64 hierarchies with the learned preconditioner (the network trained once on
            # levels 1-4 of the headline workload; its rows built inside the batched call)
            HsL = [ms.Hierarchy(2, wi.n_per_level, torch.from_numpy(wi.points).cuda(), wi.h,
                                precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED, wendland_d=2,
                                wendland_k=1, nu=wi.nu) for wi in wsb]
            for Hi in HsL:
                Hi.precond_params(params)
            hl = [Hi.handle for Hi in HsL]
            ms.ms_fit_batch(hl, fsb, REL_TOL)
            for Hi in HsL:  # new weights: the next batched call builds the rows again, inside the timing
                Hi.precond_params(params)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev[0].record(stream)
            AbL, stbL = ms.ms_fit_batch(hl, fsb, REL_TOL)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t_bl = ev[0].elapsed_time(ev[1])
            worstL = max(float(torch.linalg.norm(al - ai) / torch.linalg.norm(ai)) for al, ai in zip(AbL, Ab))
            out["batch_hierarchies"]["learned_batched_ms"] = t_bl
            out["batch_hierarchies"]["learned_kernel_ms"] = stbL[0]["fit_ms"]
            out["batch_hierarchies"]["learned_rel_residual_max"] = max(max(s["rel_residual"]) for s in stbL)
            out["batch_hierarchies"]["learned_rel_diff_vs_plain_batched_max"] = worstL
            for Hi in HsL:
                Hi.close()
            del fsb, Ab, AbL

        # the paper's own experiment (Section 5: grids (2^l+1)^2, phi_{3,1}, nu = 4, Franke data), plain
        # FP64 as the paper runs it, against Figure 4's A100 times (context: other hardware, tolerance
        # not reported there)
        if not args.no_paper:
            paper_s = {7: 0.974, 8: 1.485, 9: 4.479, 10: 20.111, 11: 92.642}
            rows = []
            for Lp in (7, 8, 9, 10, 11):
                wp = inputs.franke_grid_hierarchy(Lp)
                pp, fp = torch.from_numpy(wp.points).cuda(), torch.from_numpy(wp.f).cuda()
                best = None
                for _ in range(2):
                    rp = step(ms.MS_PREC_FP64, wl=wp, pts_=pp, f_=fp)
                    if best is None or rp["total"] < best["total"]:
                        best = rp
                rows.append({"levels": Lp, "points": int(wp.N), "step_ms": best["total"],
                             "fit_ms": best["stats"]["fit_ms"], "build_ms": best["info"]["build_ms"],
                             "cg_iterations": best["stats"]["cg_iterations"],
                             "paper_a100_solve_s": paper_s[Lp],
                             "paper_over_fit": paper_s[Lp] * 1e3 / best["stats"]["fit_ms"]})
                del pp, fp
            out["paper_grids_fp64"] = rows

        # the 3-D configuration (uniform random points, 6 levels, 4.68M points): FP64 CSR against
        # MIXED with the FP32 matrix-free inner mat-vec (levels beyond FP32 switch to FP64 CG)
        if args.cfg3:
            w3 = inputs.random3d_hierarchy(L=6)
            p3, f3 = torch.from_numpy(w3.points).cuda(), torch.from_numpy(w3.f).cuda()
            o3 = {"workload": "d=3 uniform random, N_j=125*8^(j-1), 6 levels (4,681,125 points), "
                              "delta_j=3h_j, phi_{3,1}, 30 Gaussians"}
            # the network for 3-D patches (48 inputs), trained on levels 1-4 of this hierarchy
            Ht3 = ms.Hierarchy(3, w3.n_per_level, p3, w3.h, precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED,
                               wendland_d=3, wendland_k=1, nu=w3.nu)
            o3["train"] = Ht3.train_precond([0, 1, 2, 3], epochs=max(10, args.train_epochs // 4))
            params3 = Ht3.precond_params()
            Ht3.close()
            for tag, kw in (("fp64_csr", {"prec": ms.MS_PREC_FP64}),
                            ("mixed_matrix_free", {"prec": ms.MS_PREC_MIXED, "op": ms.MS_OP_MATRIX_FREE}),
                            ("mixed_csr", {"prec": ms.MS_PREC_MIXED}),
                            ("learned_pcg_csr", {"prec": ms.MS_PREC_MIXED, "precond": ms.MS_PRECOND_LEARNED})):
                extra = {"op": kw["op"]} if "op" in kw else {}
                try:
                    r3 = step(kw["prec"], kw.get("precond", ms.MS_PRECOND_NONE), wl=w3, pts_=p3, f_=f3, **extra)
                    o3[tag] = {"step_ms": r3["total"], "fit_ms": r3["stats"]["fit_ms"],
                               "build_ms": r3["info"]["build_ms"], "cg_iterations": r3["stats"]["cg_iterations"],
                               "fp64_fallbacks": r3["stats"]["fp64_fallbacks"],
                               "rel_residual_max": max(r3["stats"]["rel_residual"])}
                except ms.MsError as e:
                    o3[tag] = {"error": str(e)[:160]}
            out["random3d"] = o3
            del p3, f3

        # end to end through the host-pointer C ABI (H2D of points, f, queries; D2H of alpha, values)
        e2e = []
        for i in range(max(2, args.steps // 2) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Hh = ms.Hierarchy(2, n, w.points, w.h, precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED,
                              wendland_d=2, wendland_k=1, nu=w.nu)
            Hh.precond_params(params)
            a_h, _ = Hh.fit(w.f, REL_TOL)
            s_h = Hh.evaluate(a_h, Qh)
            Hh.close()
            if i > 0:
                e2e.append(1000.0 * (time.perf_counter() - t0))
        h2d = w.points.nbytes + w.f.nbytes + Qh.nbytes + params.nbytes
        d2h = a_h.nbytes + s_h.nbytes
        out["e2e"] = {"value": statistics.mean(e2e), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}

        if not args.no_cpu:
            cb = cpu_baseline(args.cpu_levels, 4096)
            scale = w.N / cb["N"]
            out["cpu_baseline"] = {"value": 1000.0 * cb["times"][0] * scale, "unit": "ms", "cores": 1,
                                   "kind": "oracle",
                                   "sample": (f"oracle fit_sequential + evaluate on the first {args.cpu_levels} "
                                              f"levels ({cb['N']} points, 4096 queries) took "
                                              f"{cb['times'][0]:.2f} s single-threaded; scaled by points "
                                              f"({w.N}/{cb['N']})")}

        line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": workload_label(args.levels),
                           "path": "learned-PCG MIXED: FP32 CSR mat-vecs, FP64 dots/refinement, learned FSAI",
                           "rel_tol": REL_TOL, "queries": args.query_side ** 2,
                           "step": "build_hierarchy + precond rows + fit + evaluate, inputs resident in HBM",
                           "l2": "flushed between steps (256 MB write); CSR working set >> L2",
                           "parallelism": f"replicas x{ws}"},
                "wall_s_timed": t_wall, "gpu_launches": launches, "clocks": clk, **out}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
