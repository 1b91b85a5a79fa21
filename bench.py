#!/usr/bin/env python3
"""Benchmark of the per-evaluation likelihood hot path on one segment batch.

Workload (default): one gap-free segment, N = 8192 samples at 2048 Hz, a
batch of K = 4096 residuals r_k = d - h(theta_k) (coloured noise + a
Newtonian chirp at SNR 10, templates from the chirp priors), FP32 residuals,
FP64 logL.  The factor (covariance build, Cholesky, log det, operator
slices) runs once before timing and is reported separately; one step is one
td_loglike_batch call over the resident batch (slice the residuals, the
tensor-core whitening with its chi2 epilogue, the logL reduction).

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank evaluates
its own batch on the same segment shape (independent work, no collective on
the data path); value = evaluations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logL evals/s and p50/p99 latency at N=8192,16384 gapped; |ΔlogL| vs FP64 oracle"
UNIT = "logL evals/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="bf16x6", choices=["bf16x6", "bf16x10", "bf16x3", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-grouped", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=20.0,
                   help="timed seconds of the serving fleet's open-loop stream (after a 2 s warm-up)")
    p.add_argument("--core", action="store_true",
                   help="the headline workload, its end-to-end figure and the CPU baseline only (profiling)")
    p.add_argument("--mix-segments", type=int, default=64,
                   help="segments of the grouped mix (fewer: a small case for profiling)")
    p.add_argument("--factor-n", default="16384,32768",
                   help="segment lengths of the factor block (3 gaps of 512 each)")
    p.add_argument("--only", default=None,
                   choices=["grouped", "serving", "gapped3", "refine", "gsce", "small", "factor"],
                   help="run one extra workload alone and print its JSON object (profiling; not the bench line)")
    return p.parse_args()


def tc_sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def tf32_tflops():
    """cuBLAS TF32 GEMM rate on this GPU (8192^3, best of 5): the measured basis
    for comparing a 3xTF32 split with the bf16 splits."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        for _ in range(3):
            a @ b
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class Clocks:
    """nvidia-smi sampling (every 20 ms, timestamped); mark() brackets the timed
    region and stop() keeps the samples taken inside it (all samples if none)."""

    def __init__(self):
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def mark(self, begin):
        import datetime
        if begin:
            self.t0 = datetime.datetime.now()
        else:
            self.t1 = datetime.datetime.now()

    def stop(self):
        import datetime
        if self.proc is None:
            return None
        time.sleep(0.05)   # the sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(f[2]), float(f[3]), [nm for nm, v in zip(names, f[6:10])
                                                             if v.lower() == "active"]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": float(max(r[2] for r in use)),
                "reasons": sorted({nm for r in use for nm in r[3]}), "samples": len(use),
                "samples_in_timed_region": len(inside)}


def make_workload(rank: int):
    from paper_2603_06010_b300 import inputs
    c = inputs.GAPFREE_N8192_K4096
    seg = inputs.make_segment(c["n"], c["fs"], c["seed"])
    R = inputs.residual_batch(seg, c["K"], c["seed"] + 1 + 7919 * rank)
    return c, seg, R


def profile_traffic(name):
    """DRAM bytes per launch from a committed ncu summary under profiles/ (None if absent)."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            m = re.search(r"DRAM traffic per launch: ([0-9.]+) MB", f.read())
        return float(m.group(1)) * 1e6 if m else None
    except OSError:
        return None


def golden_chi2_rel(chi2_host):
    """max relative chi2 error on the stored oracle columns."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "full_size.json")) as f:
            g = json.load(f)["gapfree_n8192_k4096"]
        exp = np.array(g["chi2"])
        return float(np.max(np.abs(chi2_host[g["columns"]] - exp) / exp))
    except Exception:
        return None


def golden_dlogl(logL_host):
    """max |dlogL| on the stored oracle columns (rank 0's batch only)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "full_size.json")) as f:
            g = json.load(f)["gapfree_n8192_k4096"]
        cols = g["columns"]
        return float(np.max(np.abs(logL_host[cols] - np.array(g["logL"]))))
    except Exception:
        return None


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


REF_COLS = 128   # residual columns per oracle sample (both the baseline leg and the reference arm)


def cpu_baseline(seg, R, budget_s=12.0):
    """The CPU FP64 oracle, as it stands, on a bounded sample of the batch."""
    import oracle
    o = oracle.OracleSegment(seg.acf, seg.mask)
    ncols = REF_COLS
    sample = R[:ncols]
    secs, threads = oracle.time_per_eval_path(o, sample, threads=os.cpu_count(), min_seconds=budget_s)
    # one column on one thread, the form of the paper's per-evaluation CPU timings: in
    # a child process whose BLAS starts with one thread (no run-time thread control needed)
    one_s = None
    try:
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import sys, numpy as np; sys.path.insert(0, sys.argv[1]); import oracle; "
                "from paper_2603_06010_b300 import inputs; c = inputs.GAPFREE_N8192_K4096; "
                "s = inputs.make_segment(c['n'], c['fs'], c['seed']); R = inputs.residual_batch(s, 1, c['seed'] + 1); "
                "o = oracle.OracleSegment(s.acf, s.mask); t, _ = oracle.time_per_eval_path(o, R, min_seconds=2.0); "
                "print(t)")
        res = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=300)
        one_s = float(res.stdout.strip().splitlines()[-1])
    except Exception:
        one_s = None
    return {"value": ncols / secs, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{ncols} of the {R.shape[0]} residual columns, N'={o.n_kept}; "
                      f"factor excluded; LAPACK dtrtrs + FP64 chi2 on {threads} threads, "
                      f"repeated for >= {budget_s:.0f} s",
            "single_thread_single_column_ms": one_s * 1e3 if one_s is not None else None,
            "single_thread": "child process with OPENBLAS/OMP/MKL_NUM_THREADS=1, one column, >= 2 s"}


def template_extra(td, torch, seg, seg_in, K):
    """Template-input form on the benchmark segment: data vector fixed, K templates per
    call; logL alone, then logL with <h,h>, <d,h>, rho_mf and rho_eff^2."""
    from paper_2603_06010_b300 import inputs
    d = seg_in.d[seg_in.kept]
    t0 = time.perf_counter()
    seg.set_data(d)
    set_ms = (time.perf_counter() - t0) * 1e3
    H = torch.from_numpy(inputs.template_batch(seg_in, K, 7070)).cuda()
    outs = {k: torch.empty(K, dtype=torch.float64, device="cuda") for k in ("logL", "hh", "dh", "rho_mf", "rho_eff2")}
    res = {}
    for name, kw in (("logL_only", {}), ("with_snr", {k: outs[k] for k in ("hh", "dh", "rho_mf", "rho_eff2")})):
        for _ in range(3):
            seg.template_into(H, outs["logL"], **kw)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            seg.template_into(H, outs["logL"], **kw)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 10
        res[name] = {"ms_per_call": ms, "templates_per_s": K / (ms / 1e3)}
    rho = outs["rho_mf"].cpu().numpy()
    res.update({"note": f"K={K} chirp templates per call on the gap-free N=8192 segment; <d,d> once "
                        "(td_set_data); SNR outputs whiten the templates in the same batch (2K columns)",
                "set_data_ms": set_ms, "rho_mf_max": float(np.max(rho))})
    # the same call with the detector projection and placement on the device
    # (td_project_batch): polarizations of lw = N/2 samples, antenna factors and
    # sample offsets per template
    lw = seg_in.n // 2
    hp, hc, fp, fc, off = inputs.polarization_batch(seg_in, K, lw, 7071)
    hpd, hcd = torch.from_numpy(hp).cuda(), torch.from_numpy(hc).cuda()
    fpd, fcd, offd = torch.from_numpy(fp).cuda(), torch.from_numpy(fc).cuda(), torch.from_numpy(off).cuda()
    for _ in range(3):
        seg.project_into(hpd, hcd, fpd, fcd, offd, outs["logL"])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(10):
        seg.project_into(hpd, hcd, fpd, fcd, offd, outs["logL"])
    b.record()
    torch.cuda.synchronize()
    seg.check()
    ms = a.elapsed_time(b) / 10
    res["projected"] = {"ms_per_call": ms, "templates_per_s": K / (ms / 1e3), "waveform_samples": lw,
                        "h2d_bytes_per_template_3det": 2 * lw * 4,
                        "h2d_bytes_per_template_3det_detector_frame": 3 * seg_in.n_kept * 4,
                        "note": "td_project_batch: F+ h+ + Fx hx placed at an integer sample offset and "
                                "gathered on the device; a network's detectors share one upload of the "
                                "two polarizations instead of one detector-frame template each"}
    return res


def gapped_joint_extra(td, torch):
    """The gapped three-detector workload: N=16384 at 2048 Hz with 3 gaps of 512
    (N'=14848) per detector, PSD scales 1.0/1.3/2.1, K=1024 residuals each, the
    joint logL summed over detectors in the same captured launch."""
    from paper_2603_06010_b300 import inputs
    c = inputs.GAPPED_N16384_3DET
    t0 = time.perf_counter()
    segs, Rs, outs, gold = [], [], [], None
    for d, sc in enumerate(c["scales"]):
        si = inputs.make_segment(c["n"], c["fs"], c["seed"] + 10 * d, n_gaps=c["n_gaps"], gap_len=c["gap_len"],
                                 scale=sc)
        R = inputs.residual_batch(si, c["K"], c["seed"] + 10 * d + 1)
        seg = td.Segment(si.acf, si.mask)
        seg.release_fp64()
        segs.append(seg)
        Rs.append(torch.from_numpy(R).cuda())
        outs.append(torch.empty(c["K"], dtype=torch.float64, device="cuda"))
    factor_s = time.perf_counter() - t0
    joint = torch.empty(c["K"], dtype=torch.float64, device="cuda")
    g = td.Group(segs, Rs, outs)
    g.set_joint(joint)
    for _ in range(3):
        g.graph_launch()
    torch.cuda.synchronize()
    reps = 20
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for ea, eb in evs:
        flush.zero_()                      # L2 flush between launches (not timed)
        ea.record()
        g.graph_launch()
        eb.record()
    torch.cuda.synchronize()
    g.check()
    lat = np.array([ea.elapsed_time(eb) for ea, eb in evs])
    ms = float(lat.mean())
    del flush
    dlogl = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "full_size.json")) as f:
            gg = json.load(f)["gapped_n16384_3det"]
        jl = joint.cpu().numpy()
        dlogl = float(np.max(np.abs(jl[gg["columns"]] - np.array(gg["joint_logL"]))))
    except (OSError, KeyError):
        pass
    nk = segs[0].n_kept
    g.close()
    # factor checkpoint and resume: detector 0 (its operator) to a file and back,
    # against the factor it replaces; the loaded segment must give the same bits
    import tempfile
    ck = {}
    with tempfile.TemporaryDirectory() as tmpd:
        path = os.path.join(tmpd, "det0.ckpt")
        t1 = time.perf_counter()
        segs[0].save(path)
        ck["save_s"] = time.perf_counter() - t1
        ck["file_bytes"] = os.path.getsize(path)
        t1 = time.perf_counter()
        loaded = td.Segment.load(path)
        ck["load_s"] = time.perf_counter() - t1
        a_ll = torch.empty(c["K"], dtype=torch.float64, device="cuda")
        b_ll = torch.empty(c["K"], dtype=torch.float64, device="cuda")
        segs[0].loglike_into(Rs[0], a_ll)
        loaded.loglike_into(Rs[0], b_ll)
        torch.cuda.synchronize()
        ck["same_bits"] = bool(torch.equal(a_ll, b_ll))
        loaded.close()
    ck["factor_s_per_detector"] = factor_s / len(segs)
    ck["note"] = ("td_segment_save / td_segment_load of one N'=14848 detector (operator slices; FP64 factor "
                  "released), file in a temporary directory, against the FP64 factor it replaces")
    for sg in segs:
        sg.close()
    return {"note": "3 detectors, N=16384 with 3 gaps of 512 (N'=14848), K=1024 each; one captured grouped "
                    "launch writes the three detector logL and their sum",
            "ms_per_launch": ms, "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                "p99": float(np.percentile(lat, 99))},
            "l2": "flushed between launches (256 MB write)",
            "joint_evals_per_s": c["K"] / (ms / 1e3),
            "detector_evals_per_s": 3 * c["K"] / (ms / 1e3),
            "algorithmic_tflops": 3 * float(nk) ** 2 * c["K"] / (ms / 1e3) / 1e12,
            "max_abs_dlogL_joint_vs_oracle": dlogl, "factor_s": factor_s, "checkpoint": ck}


def grouped_extra(td, torch, count=64):
    """The 64-segment uneven mix (N log-uniform in [512, 32768]) in one grouped launch
    (count < 64: the mix's first segments, a small case for profiling)."""
    from paper_2603_06010_b300 import inputs
    specs = inputs.mix64_segments(count=count)
    rng = np.random.default_rng(4040)
    segs, Rs, outs = [], [], []
    t0 = time.perf_counter()
    for sp in specs:
        n = int(sp["n"])
        acf = inputs.acf_from_psd(n, sp["fs"], a=sp["a"], floor=sp["floor"])
        segs.append(td.Segment(acf, factor=False))
        R = (rng.standard_normal((sp["K"], n)) * np.sqrt(acf[0])).astype(np.float32)
        Rs.append(torch.from_numpy(R).cuda())
        outs.append(torch.empty(sp["K"], dtype=torch.float64, device="cuda"))
    td.factor_many(segs)   # gap-free: Levinson-Durbin operator build, batched
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    g = td.Group(segs, Rs, outs)
    tuned_ms = g.tune()
    bn, sf, ni = g.shape()
    for _ in range(3):
        g.graph_launch()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    clocks = Clocks()   # launches of ~17 ms back to back: the power cap sets the SM clock
    clocks.start()
    try:
        g.clock()   # clears the product kernels' clock sums (autotuner and warm-up launches)
    except Exception:
        pass
    clocks.mark(True)
    a.record()
    for _ in range(reps):
        g.graph_launch()
    b.record()
    torch.cuda.synchronize()
    clocks.mark(False)
    clk = clocks.stop()
    g.check()
    kern_mhz = g.clock()
    ms = a.elapsed_time(b) / reps
    cols = sum(int(r.shape[0]) for r in Rs)
    flops = sum(float(s.n_kept) ** 2 * int(r.shape[0]) for s, r in zip(segs, Rs))
    g.close()
    pk, basis = peaks()
    achieved = flops / (ms / 1e3) / 1e12
    sm_mhz = kern_mhz
    clock_peak = 8192.0 * tc_sms() * sm_mhz * 1e6 / 6 / 1e12
    traffic = profile_traffic("k_tc_cdo_mix64_grouped_dram.md") if count == 64 else None
    roof = {"achieved": achieved, "unit": "TFLOP/s", "sm_mhz_in_kernel": kern_mhz,
            "traffic": traffic, "traffic_over_algorithmic": traffic / 31.7e9 if traffic else None,
            "traffic_source": "profiles/k_tc_cdo_mix64_grouped_dram.md (ncu dram__bytes_read.sum + "
                              "dram__bytes_write.sum of the six-product launch, one pass); algorithmic: operator "
                              "and residual slices once, 31.7 GB" if traffic else None,
            "frac_burst": achieved / (pk["bf16_tflops"] / 6),
            "frac_sustained": achieved / (pk["bf16_tflops_sustained"] / 6),
            "frac_clock_normalized": achieved / clock_peak if clock_peak else None,
            "peak_basis": f"{basis} bf16 dense burst {pk['bf16_tflops']} / sustained "
                          f"{pk['bf16_tflops_sustained']} TF/s over 6 split products; clock-normalised: 8192 bf16 "
                          "flop/clock/SM x SMs x the SM MHz the product kernels measured (clock64 over globaltimer) / 6 (the 24 segments below 2048 kept "
                          "samples take ten products: 0.6% of the launch)"}
    dlogl = None
    try:   # the four shortest segments against the CPU oracle
        import oracle
        worst = 0.0
        for i in sorted(range(len(specs)), key=lambda j: specs[j]["n"])[:4]:
            sp = specs[i]
            acf = inputs.acf_from_psd(int(sp["n"]), sp["fs"], a=sp["a"], floor=sp["floor"])
            o = oracle.OracleSegment(acf)
            R = Rs[i].cpu().numpy()
            exp = oracle.loglike_from_chi2(o.chi2(R), o.logdet, o.n_kept)
            worst = max(worst, float(np.max(np.abs(outs[i].cpu().numpy() - exp))))
        dlogl = worst
    except Exception as ex:
        dlogl = repr(ex)
    return {"note": f"{len(specs)} segments, N log-uniform in [512, 32768], K uniform in [16, 512], own PSD each "
                    "(operators by the Levinson-Durbin build); one captured-graph grouped launch",
            "segments": len(segs), "columns": cols, "ms_per_launch": ms, "evals_per_s": cols / (ms / 1e3),
            "algorithmic_tflops": achieved, "roofline": roof, "clocks": clk, "tile_rows": bn, "chunk_factor": sf,
            "work_items": ni, "autotune_best_ms": tuned_ms, "factor_s": factor_s,
            "max_abs_dlogL_vs_oracle_4_shortest": dlogl}


def factor_extra(td, torch, with_fp64_cores=True, sizes=(16384, 32768)):
    """The factor C = L L^T with L^{-1} and the operator slices (once per segment):
    gapped N=16384 (3 gaps of 512, N'=14848) and gapped N=32768 (N'=31232) on the
    tensor-core route, and the N=16384 segment on the FP64 CUDA-core route beside it."""
    from paper_2603_06010_b300 import inputs
    out = {"note": "td_factor: blocks of 128, the block factor and its inverse in double-float, panel and trailing "
                   "updates as FP64-accurate split bf16 products on the tensor cores (six slices); wall time "
                   "of the synchronous call (covariance gather, factor, L^-1, log det, operator slices)",
           "runs": []}
    for n in sizes:
        seed = {16384: 3003, 32768: 3004}.get(n, 3000 + n % 997)
        si = inputs.make_segment(n, 2048.0, seed, n_gaps=3, gap_len=512)
        runs = {}
        for route in (("tensor", 0), ("fp64_cores", td.TD_FACTOR_FP64_CORES)):
            if route[0] == "fp64_cores" and (not with_fp64_cores or n > 16384):
                continue
            seg = td.Segment(si.acf, si.mask, factor=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if route[1]:
                td.factor_many([seg], flags=route[1])
            else:
                seg.factor()
            torch.cuda.synchronize()
            runs[route[0]] = {"s": time.perf_counter() - t0, "logdet": seg.logdet, "n_kept": seg.n_kept}
            seg.close()
        nk = runs["tensor"]["n_kept"]
        r = {"N": n, "gaps": 3, "n_kept": nk, "tensor_s": runs["tensor"]["s"],
             "fp64_equiv_tflops": (2.0 / 3.0) * float(nk) ** 3 / runs["tensor"]["s"] / 1e12}
        if "fp64_cores" in runs:
            r["fp64_cores_s"] = runs["fp64_cores"]["s"]
            r["speedup"] = runs["fp64_cores"]["s"] / runs["tensor"]["s"]
            r["logdet_rel_diff"] = abs(runs["tensor"]["logdet"] - runs["fp64_cores"]["logdet"]) / abs(
                runs["fp64_cores"]["logdet"])
        out["runs"].append(r)
    return out


def refine_extra(td, torch, seg, R, K):
    """The refinement step on the benchmark batch: per first-pass precision, one pass
    against one pass + refinement (time per call, max |dlogL| on the stored oracle columns)."""
    stream = torch.cuda.current_stream()
    logL = torch.empty(K, dtype=torch.float64, device="cuda")
    chi2 = torch.empty(K, dtype=torch.float64, device="cuda")
    runs = []
    for pname, prec, refine in (("bf16x3", td.TD_PREC_BF16X3, 0), ("bf16x3", td.TD_PREC_BF16X3, 1),
                                ("bf16x3", td.TD_PREC_BF16X3, 2), ("bf16x6", td.TD_PREC_BF16X6, 0),
                                ("bf16x6", td.TD_PREC_BF16X6, 1), ("bf16x6", td.TD_PREC_BF16X6, 2),
                                ("bf16x10", td.TD_PREC_BF16X10, 0)):
        o = td.options(precision=prec, refine=refine)
        for _ in range(3):
            seg.loglike_into(R, logL, o, chi2=chi2)
        torch.cuda.synchronize()
        seg.check()
        dll = golden_dlogl(logL.cpu().numpy())
        crel = golden_chi2_rel(chi2.cpu().numpy())
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(5):
            seg.loglike_into(R, logL, o)
        eb.record(stream)
        torch.cuda.synchronize()
        ms = ea.elapsed_time(eb) / 5
        runs.append({"precision": pname, "refine": refine, "call_ms": ms, "evals_per_s": K / (ms / 1e3),
                     "max_abs_dlogL_vs_oracle": dll, "max_chi2_rel_vs_oracle": crel})
    return {"note": "one pass vs one pass + refinement: refine 1 = w~ at the precision, s = r - L w~ by ten "
                    "split products of L's own slices, delta = L^{-1} s at the precision; refine 2 = s formed "
                    "to FP64 accuracy (six-slice split products of L and w~ per 128-column chunk, FP64 "
                    "accumulation), delta with at least six products; calls back to back, inputs (134 MB) and "
                    "the operator larger than L2", "runs": runs}


def gsce_extra(td, torch, seg_in, R, K):
    """Gohberg-Semencul path (gap-free segments): the benchmark batch and small batches at
    N=8192, then a long segment (N=32768) beside the dense path on the same segment."""
    from paper_2603_06010_b300 import inputs
    stream = torch.cuda.current_stream()

    def timed(seg, Rs, opt, reps):
        out = torch.empty(Rs.shape[0], dtype=torch.float64, device="cuda")
        for _ in range(3):
            seg.loglike_into(Rs, out, opt)
        torch.cuda.synchronize()
        seg.check()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(reps):
            seg.loglike_into(Rs, out, opt)
        eb.record(stream)
        torch.cuda.synchronize()
        return ea.elapsed_time(eb) / reps, out

    gs = td.TD_PATH_GSCE
    seg = td.Segment(seg_in.acf, factor=False)
    t0 = time.perf_counter()
    seg.gs_prepare()
    prep = time.perf_counter() - t0
    ms, out = timed(seg, R, td.options(path=gs), 5)
    res = {"note": "chi2 = (|L_x^T r|^2 - |R_x r|^2)/x_0 with x = C^-1 e_1 (Levinson-Durbin, FP64), the two "
                   "triangular Toeplitz products as FP32 circular convolutions of length M = 2^m >= 2N, one "
                   "8-CTA cluster per column pair; call_ms of back-to-back calls",
           "gapfree_n8192": {"prepare_s": prep, "K": K, "call_ms": ms, "evals_per_s": K / (ms / 1e3),
                             "max_abs_dlogL_vs_oracle": golden_dlogl(out.cpu().numpy()),
                             "small_batches": []}}
    for k in (1, 8, 64):
        mk, _ = timed(seg, R[:k].contiguous(), td.options(path=gs), 20)
        res["gapfree_n8192"]["small_batches"].append({"K": k, "call_ms": mk, "evals_per_s": k / (mk / 1e3)})
    seg.close()
    n, fs = 32768, 4096.0
    acf = inputs.acf_from_psd(n, fs)
    Rl = torch.from_numpy(inputs.noise_residuals(n, fs, 512, 11)).cuda()
    long_seg = td.Segment(acf, factor=False)
    t0 = time.perf_counter()
    long_seg.gs_prepare()
    prep = time.perf_counter() - t0
    dense_seg = td.Segment(acf, factor=False)   # the dense operator of the same segment, for comparison
    t0 = time.perf_counter()
    td.factor_many([dense_seg])
    fac = time.perf_counter() - t0
    runs = []
    for k in (1, 64, 512):
        Rk = Rl[:k].contiguous()
        mg, og = timed(long_seg, Rk, td.options(path=gs), 10)
        md, od = timed(dense_seg, Rk, td.options(), 10)
        runs.append({"K": k, "gsce_call_ms": mg, "dense_call_ms": md,
                     "max_abs_dlogL_gsce_vs_dense": float((og - od).abs().max().item())})
    long_seg.close()
    dense_seg.close()
    res["gapfree_n32768"] = {"prepare_s": prep, "dense_operator_build_s": fac, "runs": runs,
                             "dense": "td_factor_many operator, default options (BF16X6, automatic path)"}
    return res


def host_mem_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemTotal:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def fp64_per_request(td, torch, fleet, pools, served):
    """The plain per-request FP64 solve the serving workload is compared with:
    the FP64 factor L and the blocked FP64 forward substitution, one request
    at a time with no batching, on the first gapped segment of each length.
    Its service time per (N, K), and over the phase-1 requests (their N and K)
    the rate and latency it would give without any queueing."""
    from paper_2603_06010_b300 import inputs
    segs_p, Ks_p = served[0], served[1]
    o64 = td.options(precision=td.TD_PREC_FP64)
    svc = {}
    for n in (4096, 8192, 16384, 32768):
        i = next(j for j, sp in enumerate(fleet) if sp["n"] == n and sp["gaps"] > 0)
        sp = fleet[i]
        seg = td.Segment(inputs.acf_from_psd(sp["n"], sp["fs"]), sp["mask"])
        for k in (1, 8, 64, 512):
            R = pools[i][:k].contiguous()
            out = torch.empty(k, dtype=torch.float64, device="cuda")
            seg.loglike_into(R, out, o64)
            torch.cuda.synchronize()
            seg.check()
            reps = 5 if n * k <= 32768 * 8 else 2
            times = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                seg.loglike_into(R, out, o64)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            svc[(n, k)] = float(np.median(times))
        seg.close()
    t = np.array([svc[(fleet[int(sg)]["n"], int(k))] for sg, k in zip(segs_p, Ks_p)])
    mean_ms = float(t.mean())
    return {"note": "plain FP64 solve per request (FP64 L, blocked forward substitution on the FP64 cores, "
                    "no batching), on the first gapped segment of each N; service time per (N, K), median "
                    "of repeats; then over the phase-1 requests (their N and K, no queueing): mean service "
                    "time, the request rate one GPU could sustain, evals/s and latency percentiles",
            "service_ms": {f"N={n} gapped": {f"K={k}": svc[(n, k)] for k in (1, 8, 64, 512)}
                           for n in (4096, 8192, 16384, 32768)},
            "mean_service_ms": mean_ms, "max_requests_per_s": 1e3 / mean_ms,
            "evals_per_s": float(np.mean(Ks_p)) * 1e3 / mean_ms,
            "p50_ms_no_queue": float(np.percentile(t, 50)), "p99_ms_no_queue": float(np.percentile(t, 99))}


def fp64_served(td, torch, fleet, pools, phases=((2000.0, 0.1), (15.0, 8.0)), seed=5150):
    """The plain per-request FP64 solve actually served: open-loop Poisson
    arrivals (segment length uniform over the four N, one gapped segment of
    each, K uniform over {1, 8, 64, 512}), requests taken one at a time in
    arrival order on one stream, each the FP64 forward substitution with the
    FP64 factor, no batching.  Latency = completion - arrival (queueing
    included), per phase: the workload's 2000 req/s for a short burst, and a
    rate this server can sustain."""
    from paper_2603_06010_b300 import inputs
    o64 = td.options(precision=td.TD_PREC_FP64)
    Ns = (4096, 8192, 16384, 32768)
    segs, srcs = {}, {}
    for n in Ns:
        i = next(j for j, sp in enumerate(fleet) if sp["n"] == n and sp["gaps"] > 0)
        sp = fleet[i]
        segs[n] = td.Segment(inputs.acf_from_psd(sp["n"], sp["fs"]), sp["mask"])
        srcs[n] = pools[i]
    outs = {k: torch.empty(k, dtype=torch.float64, device="cuda") for k in (1, 8, 64, 512)}
    for n in Ns:   # warm-up: every (N, K) once
        for k in (1, 8, 64, 512):
            segs[n].loglike_into(srcs[n][:k].contiguous(), outs[k], o64)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    res = {}
    for rate, secs in phases:
        n_req = max(1, int(rate * secs))
        arrive = np.cumsum(rng.exponential(1.0 / rate, n_req))
        req_n = rng.choice(Ns, n_req)
        req_k = rng.choice((1, 8, 64, 512), n_req)
        lat = np.empty(n_req)
        t0 = time.perf_counter()
        for q in range(n_req):
            while time.perf_counter() - t0 < arrive[q]:
                pass
            n, k = int(req_n[q]), int(req_k[q])
            segs[n].loglike_into(srcs[n][:k], outs[k], o64)
            torch.cuda.synchronize()
            lat[q] = (time.perf_counter() - t0 - arrive[q]) * 1e3
        span = time.perf_counter() - t0
        for s in segs.values():
            s.check()
        res[f"{rate:g}_per_s"] = {"requests": n_req, "arrival_seconds": float(arrive[-1]),
                                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                  "max_ms": float(lat.max()), "completed_per_s": n_req / span,
                                  "evals_per_s": float(req_k.sum()) / span}
    for s in segs.values():
        s.close()
    res["note"] = ("plain FP64 solve served one request at a time in arrival order (FP64 L, blocked forward "
                   "substitution on the FP64 cores, no batching), open-loop Poisson arrivals, one gapped segment "
                   "per N; latency includes queueing. At the workload's rate the queue grows without bound, so "
                   "its percentiles depend on the burst length")
    return res


def serving_extra(td, torch, seconds, evict_seconds=4.0):
    """The serving workload: 200 resident segments (N uniform over 4096, 8192,
    16384, 32768 at 2048 Hz, 0-3 gaps of 512 each), open-loop Poisson arrivals
    at 2000 req/s, K uniform over {1, 8, 64, 512}, the segment uniform over the
    200.  Phase 1: the whole fleet resident (no budget).  Phase 2: the budget
    lowered by 16 GB below the fleet's operator bytes, at 50 req/s, so that
    requests evict operators to pinned host memory and reload them (pinning
    host memory runs at a few GB/s, so the spill pool is sized for what the
    phase evicts, not for the fleet)."""
    from paper_2603_06010_b300 import inputs
    fleet = inputs.serving_fleet()
    host = host_mem_bytes() or 0
    spill = int(min(24e9, 0.25 * host)) if host else 0
    srv = td.Server(max_batch_cols=2048, n_streams=4, max_kept=32768, gs_gapfree=True, host_spill_bytes=spill)
    ids, pools = [None] * len(fleet), [None] * len(fleet)
    full = {n: torch.from_numpy(inputs.serving_pool(n)).cuda() for n in (4096, 8192, 16384, 32768)}
    t0 = time.perf_counter()
    factor_by_n = {}
    # largest first: the factor's FP64 temporaries (about 17 GB at N = 32768) are
    # needed while few operators are resident
    for i in sorted(range(len(fleet)), key=lambda j: -fleet[j]["n"]):
        sp = fleet[i]
        acf = inputs.acf_from_psd(sp["n"], sp["fs"])
        t1 = time.perf_counter()
        ids[i] = srv.add_segment(acf, sp["mask"])
        srv.prefetch(ids[i])
        factor_by_n.setdefault(f"N={sp['n']} gaps>0" if sp["gaps"] else f"N={sp['n']} gap-free", []).append(
            time.perf_counter() - t1)
        kept = torch.from_numpy(inputs.kept_index(sp["mask"], sp["n"])).cuda()
        pools[i] = full[sp["n"]].index_select(1, kept).contiguous()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del full
    nk = [int(p.shape[1]) for p in pools]
    rng = np.random.default_rng(5050)

    def phase(lam, secs, warm_s=0.5):
        nreq = int(lam * (secs + warm_s))
        t = np.cumsum(rng.exponential(1.0 / lam, nreq))
        segs = rng.integers(0, len(fleet), nreq)
        Ks = rng.choice([1, 8, 64, 512], nreq)
        Rs = [pools[sg][:k] for sg, k in zip(segs, Ks)]
        outs = [torch.empty(int(k), dtype=torch.float64, device="cuda") for k in Ks]
        torch.cuda.synchronize()
        warm = int(np.searchsorted(t, warm_s))
        srv.replay(t[:warm], [ids[sg] for sg in segs[:warm]], Rs[:warm], outs[:warm])
        srv.drain()
        srv.stats(reset=True)
        tickets = srv.replay(t[warm:] - t[warm], [ids[sg] for sg in segs[warm:]], Rs[warm:], outs[warm:])
        srv.drain()
        st = srv.stats()
        lat = {}
        for sg, tk in zip(segs[warm:], tickets):
            if tk >= 0:
                sp = fleet[int(sg)]
                key = f"N={sp['n']} " + ("gapped" if sp["gaps"] else "gap-free")
                lat.setdefault(key, []).append(srv.latency_us(int(tk)) / 1e3)
        per = {k: {"requests": len(v), "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
               for k, v in sorted(lat.items())}
        res = {"arrival_rate_per_s": lam, "seconds": secs, "requests": int(st["requests_done"]),
               "refused": int(st["refused"]), "failed": int(st["failed"]), "p50_ms": st["p50_us"] / 1e3,
               "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3, "evals_per_s": st["evals_per_s"],
               "batches": int(st["batches"]), "hits": int(st["hits"]), "misses": int(st["misses"]),
               "evictions": int(st["evictions"]), "reloads": int(st["reloads"]),
               "resident_GB": st["resident_bytes"] / 1e9, "mean_K": float(np.mean(Ks[warm:])), "by_size": per}
        return res, (segs[warm:], Ks[warm:], outs[warm:], tickets)

    fleet_bytes = srv.stats()["resident_bytes"]
    p1, served = phase(2000.0, seconds, warm_s=2.0)
    # served results on the first gapped N=8192 and N=16384 segments against the
    # stored oracle logL of their request pools (a request takes the first K columns)
    checked = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "full_size.json")) as f:
            gold = {g["index"]: np.array(g["logL"]) for g in json.load(f)["serving_checked"]}
        worst, count = 0.0, 0
        segs_p, Ks_p, outs_p, tks = served
        for sg, k, o, tk in zip(segs_p, Ks_p, outs_p, tks):
            if int(sg) in gold and tk >= 0:
                worst = max(worst, float(np.max(np.abs(o.cpu().numpy() - gold[int(sg)][:int(k)]))))
                count += 1
        checked = {"requests_checked": count, "max_abs_dlogL_vs_oracle": worst,
                   "segments": [f"index {i}: N={fleet[i]['n']}, {fleet[i]['gaps']} gaps, N'={nk[i]}"
                                for i in sorted(gold)]}
    except (OSError, KeyError) as ex:
        checked = {"error": repr(ex)}
    budget = int(fleet_bytes - 16e9)
    srv.set_budget(budget)
    p2, _ = phase(50.0, evict_seconds)
    srv.close()
    fp64 = fp64_per_request(td, torch, fleet, pools, served)
    fp64["served"] = fp64_served(td, torch, fleet, pools)
    by_n = {k: {"segments": len(v), "mean_s": float(np.mean(v)), "max_s": float(np.max(v))}
            for k, v in sorted(factor_by_n.items())}
    out = {"note": "200 resident segments: N uniform over {4096, 8192, 16384, 32768} at 2048 Hz, 0-3 gaps of "
                   "512 (seeded), the reference PSD; requests open loop (native replay), K uniform over "
                   "{1, 8, 64, 512}, segment uniform over the 200; 4 streams, batches up to 2048 columns; "
                   "gap-free segments also hold the Gohberg-Semencul form (K <= 256, and any K at N = 32768, "
                   "run through it)",
           "segments": len(fleet), "operator_GB": fleet_bytes / 1e9,
           "setup_s": setup_s, "factor_s_by_kind": by_n,
           "fleet": p1, "served_accuracy": checked, "fp64_per_request": fp64,
           "eviction": dict(p2, budget_GB=budget / 1e9, host_spill_pool_GB=spill / 1e9,
                            note="budget lowered at run time to 16 GB below the fleet's operator bytes; "
                                 "evicted operators go to pinned host memory (a pool pinned at server creation) "
                                 "and come back on their next request")}
    out.update({k: p1[k] for k in ("p50_ms", "p99_ms", "evals_per_s", "requests", "refused")})
    return out


def run_reference(args):
    """The CPU FP64 oracle as the reference arm: each step evaluates the same
    128-column sample of the benchmark batch (the cpu_baseline leg's sample)
    repeatedly on all host cores, for at least max(0.25 s, 12 s / steps), so
    the timed steps together cover at least 12 s as the cpu_baseline leg does."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c, seg, R = make_workload(0)
    import oracle
    o = oracle.OracleSegment(seg.acf, seg.mask)
    sample = R[:REF_COLS]
    per_eval, threads = [], os.cpu_count()
    min_s = max(0.25, 12.0 / max(1, args.steps))
    for i in range(args.warmup + args.steps):
        secs, threads = oracle.time_per_eval_path(o, sample, threads=os.cpu_count(),
                                                  min_seconds=min_s if i >= args.warmup else 0.25)
        if i >= args.warmup:
            per_eval.append(secs)   # seconds per evaluation of the 128 columns
    step_s = np.array(per_eval)
    value = REF_COLS * len(step_s) / float(step_s.sum())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(step_s.mean()),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": c["name"], "N": c["n"], "K": c["K"], "fs": c["fs"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"the first {REF_COLS} residual columns of the K={c['K']} batch, "
                                       f"evaluated repeatedly for >= {min_s:.2f} s per step (time per evaluation "
                                       f"of the {REF_COLS} columns); factor excluded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def small_batches(td, torch, seg, R, N, prec, prec_name):
    """Batches of K = 1 ... 256 columns of the N' = 8192 workload on each tile
    shape, back to back: the product kernel alone (CUDA events around it, as
    operator GB/s and as TFLOP/s against bf16 peak / products) and the whole
    call."""
    small = []
    if prec_name not in ("bf16x6", "bf16x10"):
        return small
    stream = torch.cuda.current_stream()
    nsl = 3 if prec_name == "bf16x6" else 4
    products = 6 if prec_name == "bf16x6" else 10
    op_bytes = (N // 256) * ((N // 256) + 1) // 2 * 8 * nsl * 256 * 32 * 2   # operator slices read once
    for Ks in (1, 8, 64, 128, 256):
        Rs = R[:Ks].contiguous()
        ls = torch.empty(Ks, dtype=torch.float64, device="cuda")
        cand = [("auto", td.TD_PATH_AUTO), ("stream128", td.TD_PATH_STREAM128)]
        if Ks <= 8:
            cand.append(("stream256", td.TD_PATH_STREAM))
        if Ks >= 64:
            cand += [("smallk", td.TD_PATH_SMALLK), ("tensor128", td.TD_PATH_TENSOR128)]
        for pname, path in cand:
            o2 = td.options(precision=prec, path=path)
            for _ in range(3):
                seg.loglike_into(Rs, ls, o2)
            torch.cuda.synchronize()
            # no L2 flush: the operator streamed by every call (201 MB at N'=8192) is larger
            # than L2 (126 MB); calls are back to back, as a sampler issues them
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            for _ in range(20):
                seg.loglike_into(Rs, ls, o2)
            eb.record(stream)
            torch.cuda.synchronize()
            tot = ea.elapsed_time(eb)
            seg.profile(True)
            for _ in range(20):
                seg.loglike_into(Rs, ls, o2)
            torch.cuda.synchronize()
            kms, kn, _ = seg.profile_read()
            seg.profile(False)
            kavg = kms / max(kn, 1)
            gbs = op_bytes / (kavg / 1e3) / 1e9
            tfl = float(N) * float(N) * Ks / (kavg / 1e3) / 1e12
            tpeak = peaks()[0]["bf16_tflops"] / products
            small.append({"K": Ks, "path": pname, "kernel_ms": kavg, "call_ms": tot / 20,
                          "evals_per_s": Ks / (tot / 20 / 1e3),
                          "operator_GBps": gbs, "hbm_frac": gbs / peaks()[0]["hbm_gbs"],
                          "call_hbm_frac": op_bytes / (tot / 20 / 1e3) / 1e9 / peaks()[0]["hbm_gbs"],
                          "kernel_tflops": tfl, "tensor_frac": tfl / tpeak,
                          "call_tensor_frac": float(N) * float(N) * Ks / (tot / 20 / 1e3) / 1e12 / tpeak})
    return small


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    if args.only:
        from paper_2603_06010_b300 import build as tdbuild
        tdbuild.build()
        from paper_2603_06010_b300 import td
        torch.cuda.set_device(0)
        def only_refine():
            c, seg_in, R_host = make_workload(0)
            seg = td.Segment(seg_in.acf, seg_in.mask)
            return refine_extra(td, torch, seg, torch.from_numpy(R_host).cuda(), R_host.shape[0])
        def only_gsce():
            c, seg_in, R_host = make_workload(0)
            return gsce_extra(td, torch, seg_in, torch.from_numpy(R_host).cuda(), R_host.shape[0])
        def only_small():
            c, seg_in, R_host = make_workload(0)
            seg = td.Segment(seg_in.acf, seg_in.mask)
            return small_batches(td, torch, seg, torch.from_numpy(R_host).cuda(), R_host.shape[1],
                                 td.TD_PREC_BF16X6, "bf16x6")
        fsizes = tuple(int(x) for x in args.factor_n.split(","))
        fn = {"grouped": lambda: grouped_extra(td, torch, args.mix_segments), "serving": lambda: serving_extra(td, torch, args.serve_seconds),
              "gapped3": lambda: gapped_joint_extra(td, torch), "refine": only_refine, "gsce": only_gsce,
              "small": only_small, "factor": lambda: factor_extra(td, torch, sizes=fsizes)}[args.only]
        print(json.dumps({"only": args.only, "result": fn()}), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2603_06010_b300 import build as tdbuild
    tdbuild.build()
    from paper_2603_06010_b300 import td

    c, seg_in, R_host = make_workload(rank)
    K, N = R_host.shape[0], R_host.shape[1]
    prec = {"bf16x6": td.TD_PREC_BF16X6, "bf16x10": td.TD_PREC_BF16X10, "bf16x3": td.TD_PREC_BF16X3,
            "fp64": td.TD_PREC_FP64}[args.precision]
    opt = td.options(precision=prec)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    seg = td.Segment(seg_in.acf, seg_in.mask)
    factor_s = time.perf_counter() - t0

    R = torch.from_numpy(R_host).cuda()
    logL = torch.empty(K, dtype=torch.float64, device="cuda")
    seg.reserve(K, opt)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        seg.loglike_into(R, logL, opt)
    torch.cuda.synchronize()
    seg.check()
    logL_host = logL.cpu().numpy()
    # pinned host buffers of the end-to-end leg, allocated once at start-up as a
    # sampler would, and used once here: a pinned buffer's first host-to-device
    # copies run slowly (3.5 GB/s for the first, about 40 GB/s for the next
    # ones) and reach about 55 GB/s only some time later
    R_pin = torch.from_numpy(R_host).pin_memory()
    out_pin = torch.empty(K, dtype=torch.float64).pin_memory()
    seg.loglike_host_into(R_pin, out_pin, opt)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks()
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    seg.profile(True)
    clocks.mark(True)
    for i in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (not timed)
        ev[i][0].record(stream)
        seg.loglike_into(R, logL, opt)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    kern_ms, kern_n, kernels = seg.profile_read()
    try:   # the SM clock the product kernel ran at (its own cycle counter over the global timer)
        kern_mhz = seg.profile_clock()
    except Exception:
        kern_mhz = None
    seg.profile(False)
    seg.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    from paper_2603_06010_b300 import dist as tddist
    tot_s, all_evals = tddist.aggregate(float(step_ms.sum()) / 1e3, K * args.steps, device="cuda")
    tot_ms = tot_s * 1e3
    value = all_evals / tot_s

    # end to end through the C ABI with host buffers (pinned): td_loglike_batch_host copies the
    # residuals in, evaluates (copies of later column chunks overlap earlier evaluations) and
    # copies logL back; all of it inside the timed region
    e2e_ms = []
    for i in range(args.e2e_steps + 3):   # three untimed warm-up calls
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seg.loglike_host_into(R_pin, out_pin, opt)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            e2e_ms.append(a.elapsed_time(b))
    e2e_dlogl = golden_dlogl(out_pin.numpy()) if rank == 0 else None
    # context: the plain pinned host -> device copy rate of the same bytes (the e2e ceiling)
    Rd = torch.empty_like(R)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Rd.copy_(R_pin, non_blocking=True)
    a.record(stream)
    for _ in range(3):
        Rd.copy_(R_pin, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    h2d_gbps = 3 * R_host.nbytes / (a.elapsed_time(b) / 1e3) / 1e9
    del Rd
    e2e_s, e2e_evals = tddist.aggregate(float(np.sum(e2e_ms)) / 1e3, K * len(e2e_ms), device="cuda")
    e2e_value = e2e_evals / e2e_s

    # plain FP64 GPU solve on the same batch (the baseline the split path must beat)
    fp64 = None
    if not args.no_fp64_compare and args.precision != "fp64":
        o64 = td.options(precision=td.TD_PREC_FP64)
        seg.reserve(K, o64)
        seg.loglike_into(R, logL, o64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seg.loglike_into(R, logL, o64)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        fp64 = {"value": K / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "max_abs_dlogL_vs_oracle": golden_dlogl(logL.cpu().numpy()) if rank == 0 else None}

    # small and mid-size batches on the same segment
    small = [] if args.core else small_batches(td, torch, seg, R, N, prec, args.precision)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, basis = peaks()
    flops = float(N) * float(N) * float(K)      # N'^2 K: N'^2/2 multiply-adds per column
    kern_avg_ms = kern_ms / max(kern_n, 1)
    products = {"bf16x6": 6, "bf16x10": 10, "bf16x3": 3}.get(args.precision)
    if products:
        achieved = flops / (kern_avg_ms / 1e3) / 1e12
        peak = pk["bf16_tflops"] / products
        # DRAM bytes of this kernel and workload from the committed ncu capture (BF16X6 only)
        traffic = profile_traffic("k_tc_cdo_gapfree_n8192_k4096.md") if args.precision == "bf16x6" else None
        # the same kernel against what the tensor cores can issue at the SM clock
        # sampled during the timed region (8192 bf16 flop per clock per SM: one
        # M=128, N=256, K=16 tcgen05 MMA per 128 cycles), and against the
        # three-product basis of the BF16 split (bf16 peak / 3)
        # SM clock: the kernel's own reading (cycles over global-timer ns, summed over its CTAs),
        # else the median nvidia-smi sample
        sm_mhz = kern_mhz or (clk or {}).get("sm_mhz")
        smi_mhz = (clk or {}).get("sm_mhz")
        clock_peak = 8192.0 * tc_sms() * sm_mhz * 1e6 / products / 1e12 if sm_mhz else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_tc_cdo",
                "frac_clock_normalized": achieved / clock_peak if clock_peak else None,
                "clock_normalized_peak": clock_peak,
                "clock_normalized_mhz": sm_mhz,
                "clock_source": "in-kernel (clock64 / globaltimer over the MMA threads' spans)" if kern_mhz
                                else "nvidia-smi median",
                "frac_clock_normalized_smi": (achieved / (8192.0 * tc_sms() * smi_mhz * 1e6 / products / 1e12)
                                              if smi_mhz else None),
                "clock_normalized_basis": "8192 bf16 flop/clock/SM x SMs x SM MHz / products",
                "frac_3product_basis": achieved / (pk["bf16_tflops"] / 3),
                "traffic_source": "profiles/k_tc_cdo_gapfree_n8192_k4096.md (ncu dram__bytes_read.sum + "
                                  "dram__bytes_write.sum, one launch)" if traffic else None,
                "kernel_ms": kern_avg_ms,
                "peak_basis": f"{basis} bf16 dense burst {pk['bf16_tflops']} TF/s / {products} split products",
                "algorithmic": "N'^2 K flops per launch (N'^2/2 multiply-adds per residual column)"}
    else:
        roof = {"bound": "alu", "achieved": flops / (kern_avg_ms / 1e3) / 1e12, "peak": 1.25,
                "unit": "TFLOP/s", "frac": None, "traffic": None, "kernel": "k_f64_update + k_f64_diag",
                "kernel_ms": kern_avg_ms, "peak_basis": "nominal FP64 1.25 TF/s"}
        roof["frac"] = roof["achieved"] / roof["peak"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if products else "f64",
        "data": "synthetic",
        "config": {"workload": c["name"], "N": N, "K": K, "fs": c["fs"], "gaps": 0,
                   "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "max_abs_dlogL_vs_oracle": golden_dlogl(logL_host),
        "gpu_launches": int(kernels),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(R_host.nbytes),
                "d2h_bytes_per_step": int(K * 8), "api": "td_loglike_batch_host (pinned host buffers)",
                "max_abs_dlogL_vs_oracle": e2e_dlogl, "h2d_copy_GBps": h2d_gbps,
                "note": "bound by the host-to-device copy of the FP32 residuals"},
        "setup": {"factor_s": factor_s, "operator_bytes": seg.resident_bytes},
        "fp64_gpu_baseline": fp64,
        "small_batches": {"note": "kernel_ms = the tensor-core product kernel alone (CUDA events around it); "
                                  "call_ms = whole td_loglike_batch (slicing, product, chunk reduction, logL), "
                                  "20 calls back to back; no L2 flush (the operator read by each call is larger "
                                  "than L2); algorithmic bytes = operator slices read once (3 x 2 B per packed "
                                  "lower-triangle element); hbm_frac = of the kernel, call_hbm_frac = of the "
                                  "whole call, both of measured HBM bandwidth; kernel_tflops = N'^2 K / kernel "
                                  "time, tensor_frac / call_tensor_frac = of measured bf16 burst / products",
                          "runs": small},
        "clocks": clk,
    }
    if world == 1 and not args.core:
        line["factor"] = factor_extra(td, torch, sizes=tuple(int(x) for x in args.factor_n.split(",")))
        line["template_form"] = template_extra(td, torch, seg, seg_in, K)
        line["refinement"] = refine_extra(td, torch, seg, R, K)
        line["gsce"] = gsce_extra(td, torch, seg_in, R, K)
    if world == 1 and not args.no_grouped and not args.core:
        gj = gapped_joint_extra(td, torch)
        line["metric_configs"] = {
            "note": "the two configurations the metric names, each as evals/s, p50/p99 latency of one call "
                    "(L2 flushed before each) and max |dlogL| against stored FP64 oracle columns",
            c["name"]: {"evals_per_s": value, "latency_ms": line["latency_ms"],
                        "max_abs_dlogL_vs_oracle": line["max_abs_dlogL_vs_oracle"]},
            "gapped_n16384_3det_k1024": {"joint_evals_per_s": gj["joint_evals_per_s"],
                                         "detector_evals_per_s": gj["detector_evals_per_s"],
                                         "latency_ms": gj["latency_ms"],
                                         "max_abs_dlogL_vs_oracle": gj["max_abs_dlogL_joint_vs_oracle"]}}
        line["gapped_n16384_3det"] = gj
        line["grouped"] = grouped_extra(td, torch, args.mix_segments)
    if world == 1 and not args.core:
        try:
            line["peaks_extra"] = {"tf32_tflops_burst": tf32_tflops(),
                                   "note": "cuBLAS fp32 GEMM with TF32 enabled, 8192^3, best of 5 (measured here)"}
        except Exception as ex:
            line["peaks_extra"] = {"error": repr(ex)}
    if world == 1 and not args.no_serving and not args.core:
        line["serving"] = serving_extra(td, torch, args.serve_seconds)
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(seg_in, R_host)
        except Exception as ex:   # report, do not lose the measured line
            line["cpu_baseline"] = {"error": repr(ex)}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
