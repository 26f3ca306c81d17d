#!/usr/bin/env python
"""Benchmark of the online tensor method's hot path on one GB300 (or N replicas).

Default workload (one "step" = one pass of the whole hot path over one
synthetic input): latent Dirichlet allocation, 300,000 documents of
Poisson(300) words over a vocabulary of 100,000 (topic-word distributions
Dir(0.05) with Zipf-skewed concentrations), k = 100 topics, alpha0 = 1 -- a
synthetic stand-in for the paper's NYTimes corpus.
  whiten (randomised range finder, oversampling 20, 2 power iterations, FP64
  eigendecomposition) -> project (y_t = W^T c_t / l_t) -> means -> STGD,
  minibatch 1,024, beta_t = 1e-2/sqrt(t), theta = 1, 20 epochs (5,860 steps in
  one persistent launch) -> unwhiten (topics normalised to the simplex).
Metric: whitened samples processed by the SGD per second of whole-path time
(6,000,000 samples per step).  Inputs are resident in HBM before timing
(larger than L2); the L2 is flushed (256 MiB write) between timed steps.
``e2e`` repeats the measurement with the inputs in pinned host memory and the
copies (CSR, projection, permutations, start) and the read-back of the topics
inside the timed region.  After the timed region: the BF16 and FP8 forms of
the STGD on the same samples with their errors against the FP64 oracle, the
time to 1e-3 reconstruction error of plain FP32 STGD and of the warm-started
forms, and the FP64 oracle timed on the host cores (matrix-form STGD run to
completion).

Other workloads: --workload mmsb (the community-model pipeline, 4 x 5,000
nodes, k = 100), batched, warmstart, whitening.
``--impl reference`` times the FP64 CPU oracle on the default workload.
Multi-GPU: replicas only (one independent decomposition per rank, no
collective on the data path); value = samples of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "whitened-sample SGD throughput (samples/s) & time-to-1e-3 error vs plain FP32"
UNIT = "samples/s"
CFG = dict(workload="mmsb_4x5000_k100_b1024_fp32", n_per=5000, k=100, alpha_i=0.01, p=0.1,
           q=0.005, oversample=20, power_iters=2, b=1024, epochs=20, beta0=1e-2, theta=1.0,
           alpha0=1.0, seed=0)
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max clock
# the persistent STGD kernel the library runs for each choice of otm_sgd_set_form
SGD_KERNEL_NAME = {"auto": "sgd_grid_kernel (one cooperative launch = all STGD steps)",
                   "split": "sgd_split_kernel (one persistent launch = all STGD steps)",
                   "grid": "sgd_grid_kernel (one cooperative launch = all STGD steps)",
                   "cluster": "sgd_cluster_kernel (one cluster launch = all STGD steps)"}
PVALUE_THRESHOLD = 0.01   # significance level of the paired p-value test
# DRAM bytes (read + write) of one grid-form STGD launch on the default corpus
# (300,000 documents, k = 100, b = 1,024, 20 epochs), from one ncu capture of that
# launch (dram__bytes_read.sum + dram__bytes_write.sum); reported only while the
# kernel's source is the one that was captured (its SHA-256), else null.
SGD_GRID_TRAFFIC = {"bytes": 1732604000 + 4984320,
                    "source": "paper_1309_0787_gb300/csrc/sgd_grid.cu",
                    "sha256": "9d85a56ee0c025275d1d7c646b533cefacd2e083523fce18116f542c012ff265",
                    "capture": "ncu capture of the grid-form launch on the default corpus"}


def sgd_grid_traffic(form, c):
    """The captured DRAM bytes of the grid-form launch, for the captured workload
    and an unchanged kernel source; None otherwise."""
    if form not in ("auto", "grid") or (c["n_docs"], c["k"], c["b"], c["epochs"]) != (
            300000, 100, 1024, 20):
        return None
    try:
        with open(os.path.join(ROOT, SGD_GRID_TRAFFIC["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return SGD_GRID_TRAFFIC["bytes"] if h == SGD_GRID_TRAFFIC["sha256"] else None


def make_inputs(cfg, rank=0):
    s = cfg["seed"] + 1000 * rank
    kt = cfg["k"] + cfg["oversample"]
    g = synth.mmsb_graph(s, cfg["n_per"], cfg["k"], cfg["alpha_i"], cfg["p"], cfg["q"])
    return {"G_XA": g["G_XA"], "G_XB": g["G_XB"], "G_XC": g["G_XC"],
            "S_pairs": synth.gaussian(s + 1, cfg["n_per"], kt),
            "S_w": synth.gaussian(s + 2, cfg["n_per"], kt),
            "perm": synth.epoch_permutations(s + 3, cfg["n_per"], cfg["epochs"]),
            "V0": synth.haar_orthonormal(s + 4, cfg["k"]),
            "Pi_X": g["Pi"]["X"]}


def sgd_flops(cfg, views=3):
    """Algorithmic flops of the STGD launch: per step 2 views x 2k^2 b_s (A = V^T Y)
    + 2k^2 b_s (Y_C^T B^T) + 4k^3 (Gram term), summed over all steps."""
    n, b, k = cfg["n_per"], cfg["b"], cfg["k"]
    sizes = [min(b, n - s) for s in range(0, n, b)] * cfg["epochs"]
    per_sample = 2 * (views - 1) * k * k + 2 * k * k
    return sum(per_sample * bs + 4 * k ** 3 for bs in sizes), len(sizes)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
class GpuPath:
    def __init__(self, otm, torch, cfg, host, device):
        self.otm, self.torch, self.cfg, self.dev = otm, torch, cfg, device
        self.host = host
        self.upload()

    def upload(self, pinned=None):
        t = self.torch
        src = pinned if pinned is not None else self.host
        self.D = {x: self.otm.DeviceCSR.from_host(self.host[x], self.dev) if pinned is None else
                  self.otm.DeviceCSR(*(a.to(self.dev, non_blocking=True) for a in src[x]),
                                     self.host[x].shape)
                  for x in ("G_XA", "G_XB", "G_XC")}
        for nm in ("S_pairs", "S_w", "perm", "V0"):
            a = src[nm]
            setattr(self, nm, (t.from_numpy(np.ascontiguousarray(a)) if pinned is None else a)
                    .to(self.dev, non_blocking=True))

    def step(self, ev=None):
        otm, t, c = self.otm, self.torch, self.cfg
        k = c["k"]
        if ev:
            ev["w0"].record()
        wh = otm.whiten_community(self.D["G_XA"], self.D["G_XB"], self.D["G_XC"], self.S_pairs,
                                  self.S_w, k, c["power_iters"], c["alpha0"])
        YA = otm.project(self.D["G_XA"], wh["W"])
        YB = otm.project(self.D["G_XB"], wh["W_B"])
        YC = otm.project(self.D["G_XC"], wh["W_C"])
        yb = t.stack([otm.column_mean(YA), otm.column_mean(YB), otm.column_mean(YC)])
        V = self.V0.t().contiguous()
        if ev:
            ev["s0"].record()
        otm.sgd_run(V, YA, YB, YC, yb, self.perm, c["epochs"], c["b"], c["beta0"], c["theta"],
                    c["alpha0"])
        if ev:
            ev["s1"].record()
        out = otm.unwhiten(V, wh["Q"], wh["Cp"], c["theta"], False)
        out["Pi_hat"] = otm.membership(YA, V, c["theta"])
        return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


REF_STEPS, REF_BETA0 = 10000, 0.02   # full-batch reference run (see convergence())


def convergence(otm, torch, path, cfg, fp32_step_ms):
    """Time-to-1e-3 of the plain FP32 STGD and of the BF16 precision form on the
    bench's whitened samples.  Error = relative reconstruction error of the
    iterate (snapshot after every epoch) against a reference solution on the
    same samples: REF_STEPS full-batch FP32 steps (beta_t = REF_BETA0/sqrt(t))
    continued from the FP32 run's final iterate; its residual gradient is
    reported.  Untimed except for the BF16 run's own step time."""
    c, k = cfg, cfg["k"]
    n = c["n_per"]
    spe = (n + c["b"] - 1) // c["b"]
    wh = otm.whiten_community(path.D["G_XA"], path.D["G_XB"], path.D["G_XC"], path.S_pairs,
                              path.S_w, k, c["power_iters"], c["alpha0"])
    Y = [otm.project(path.D[x], wh[w]) for x, w in (("G_XA", "W"), ("G_XB", "W_B"),
                                                   ("G_XC", "W_C"))]
    yb = torch.stack([otm.column_mean(y) for y in Y])
    V32 = path.V0.t().contiguous()
    snap32 = otm.sgd_run(V32, *Y, yb, path.perm, c["epochs"], c["b"], c["beta0"], c["theta"],
                         c["alpha0"], snapshot_every=spe)
    q = [otm.quantize_samples(y, otm.PREC_BF16) for y in Y]
    V16 = path.V0.t().contiguous()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    snap16 = otm.sgd_run_lp(V16, *q, yb, path.perm, c["epochs"], c["b"], c["beta0"], c["theta"],
                            c["alpha0"], otm.PREC_BF16, snapshot_every=spe)
    e1.record()
    torch.cuda.synchronize()
    bf16_step_ms = e0.elapsed_time(e1) / (spe * c["epochs"])
    Vref = V32.clone()
    otm.sgd_run(Vref, *Y, yb, None, REF_STEPS, n, REF_BETA0, c["theta"], c["alpha0"])
    # residual gradient at the reference: one tiny full-batch step
    Vg = Vref.clone()
    h = 1e-3
    otm.sgd_step(Vg, *Y, yb, c["theta"], h, c["alpha0"])
    grad_rel = float(((Vref - Vg) / h).norm() / Vref.norm())
    nr = Vref.double().norm(dim=1)
    kappa = 0.5 * (1.0 + c["theta"])
    lam = (kappa * nr ** 3).contiguous()
    U = (Vref.double() / nr[:, None]).contiguous()

    def report(snaps, step_ms):
        errs = [float(otm.recon_error(snaps[i].contiguous(), U, lam, c["theta"])[0])
                for i in range(snaps.shape[0])]
        hit = next((i for i, e in enumerate(errs) if e <= 1e-3), None)
        return {"epochs_to_1e-3": None if hit is None else hit + 1,
                "seconds_to_1e-3": None if hit is None else (hit + 1) * spe * step_ms / 1e3,
                "step_ms": step_ms, "error_by_epoch": [round(e, 6) for e in errs]}
    return {"reference": f"{REF_STEPS} full-batch FP32 steps, beta0 {REF_BETA0}, "
                         "from the FP32 run's final iterate",
            "reference_grad_rel": grad_rel,
            "fp32": report(snap32, fp32_step_ms), "bf16": report(snap16, bf16_step_ms)}


def sgd_form_code(otm, name):
    return {"auto": otm.SGD_FORM_AUTO, "cluster": otm.SGD_FORM_CLUSTER,
            "grid": otm.SGD_FORM_GRID, "split": otm.SGD_FORM_SPLIT}[name]


def run_mmsb(args, rank, world, local_rank):
    import torch
    from paper_1309_0787_gb300 import otm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg = dict(CFG)
    host = make_inputs(cfg, rank)
    path = GpuPath(otm, torch, cfg, host, dev)
    otm.sgd_set_form(sgd_form_code(otm, args.sgd_form))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    samples = cfg["n_per"] * cfg["epochs"]
    flops, nsteps = sgd_flops(cfg)

    for _ in range(args.warmup):
        path.step()
    torch.cuda.synchronize()
    dist_barrier(world)

    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [{n: torch.cuda.Event(enable_timing=True) for n in ("w0", "s0", "s1", "e1")}
          for _ in range(args.steps)]
    l0 = otm.launch_count()
    torch.cuda.synchronize()
    dist_barrier(world)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                       # evict the L2 (129 MB) between steps
        path.step(ev[i])
        ev[i]["e1"].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    dist_barrier(world)
    launches = otm.launch_count() - l0
    clocks = sampler.stop()
    step_ms = [e["w0"].elapsed_time(e["e1"]) for e in ev]
    sgd_ms = [e["s0"].elapsed_time(e["s1"]) for e in ev]
    pre_ms = [e["w0"].elapsed_time(e["s0"]) for e in ev]
    t_total = sum(step_ms) / 1e3
    t_max = dist_max(t_total, world)

    # end to end: inputs in pinned host memory, copies inside the timed region
    pinned = {x: tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                       for a in (host[x].row_ptr, host[x].col, host[x].val))
              for x in ("G_XA", "G_XB", "G_XC")}
    for nm in ("S_pairs", "S_w", "perm", "V0"):
        pinned[nm] = torch.from_numpy(np.ascontiguousarray(host[nm])).pin_memory()
    h2d = sum(a.numel() * a.element_size() for x in ("G_XA", "G_XB", "G_XC") for a in pinned[x])
    h2d += sum(pinned[nm].numel() * pinned[nm].element_size()
               for nm in ("S_pairs", "S_w", "perm", "V0"))
    res_host = torch.empty(cfg["n_per"], cfg["k"], dtype=torch.float64).pin_memory()
    lam_host = torch.empty(cfg["k"], dtype=torch.float64).pin_memory()
    pi_host = torch.empty(cfg["k"], cfg["n_per"], dtype=torch.float32).pin_memory()
    d2h = res_host.numel() * 8 + lam_host.numel() * 8 + pi_host.numel() * 4
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for i in range(max(1, args.steps // 2)):
        flush.fill_(float(i))
        e_start.record()
        path.upload(pinned)
        out = path.step()
        res_host.copy_(out["comps"], non_blocking=True)
        lam_host.copy_(out["lambda"], non_blocking=True)
        pi_host.copy_(out["Pi_hat"], non_blocking=True)
        e_end.record()
        torch.cuda.synchronize()
        e2e_ms += e_start.elapsed_time(e_end)
    n_e2e = max(1, args.steps // 2)
    e2e_t = dist_max(e2e_ms / 1e3, world)

    # validation of the last membership estimate (off the timed region)
    truth = torch.from_numpy(np.ascontiguousarray(host["Pi_X"].T, dtype=np.float32)).to(dev)
    val = otm.pvalue_match(out["Pi_hat"], truth, PVALUE_THRESHOLD)
    pv = val["pvalues"].cpu().numpy()
    scores = val["scores"].cpu().numpy()

    if rank != 0:
        return None
    sgd_avg_s = statistics.mean(sgd_ms) / 1e3
    achieved = flops / sgd_avg_s / 1e12
    line = {
        "metric": METRIC, "value": world * samples * args.steps / t_max, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg["workload"], "nodes_per_part": cfg["n_per"], "k": cfg["k"],
                   "minibatch": cfg["b"], "epochs": cfg["epochs"], "sgd_steps": nsteps,
                   "samples_per_step": samples, "oversample": cfg["oversample"],
                   "power_iters": cfg["power_iters"], "alpha0": cfg["alpha0"],
                   "theta": cfg["theta"], "beta0": cfg["beta0"],
                   "nnz": [int(host[x].nnz) for x in ("G_XA", "G_XB", "G_XC")],
                   "l2": "flushed between timed steps (256 MiB write)",
                   "sgd_form": args.sgd_form,
                   "parallelism": "replicas" if world > 1 else "single"},
        "breakdown_ms": {"whiten_project_mean": statistics.mean(pre_ms),
                         "sgd_run": statistics.mean(sgd_ms),
                         "unwhiten": statistics.mean(step_ms) - statistics.mean(pre_ms)
                         - statistics.mean(sgd_ms),
                         "wall_per_step": 1e3 * wall / args.steps},
        "roofline": {"kernel": SGD_KERNEL_NAME[args.sgd_form],
                     "bound": "alu", "achieved": achieved, "peak": FP32_FMA_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_FMA_PEAK_TFLOPS,
                     "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                     "algorithmic_flops_per_launch": flops},
        "e2e": {"value": world * samples * n_e2e / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    otm.sgd_set_form(otm.SGD_FORM_AUTO)  # the full-batch reference needs the cluster form
    line["mmsb_validation"] = {
        "recovery_ratio": float(scores[0]), "average_error": float(scores[1]),
        "pvalue_threshold": PVALUE_THRESHOLD,
        "significant_pairs": int((pv <= PVALUE_THRESHOLD).sum()),
        "against": "the generator's memberships of the 5,000 X nodes"}
    line["time_to_1e-3"] = convergence(otm, torch, path, cfg, statistics.mean(sgd_ms) / nsteps)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(cfg, host)
    return line


# ----------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------
def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_sample(cfg, host, sgd_steps):
    """Time the oracle on the workload: whitening + projection + means once,
    `sgd_steps` STGD steps, unwhitening.  Returns (seconds per component)."""
    from oracle import moments as om
    from oracle import community as ocomm
    from oracle import post as opost
    from oracle import stgd as ostgd
    from oracle import whiten as ow
    k = cfg["k"]
    t0 = time.perf_counter()
    wh = ow.community_whiten_randomized(host["G_XA"], host["G_XB"], host["G_XC"], k,
                                        cfg["alpha0"], host["S_pairs"].astype(np.float64),
                                        host["S_w"].astype(np.float64), cfg["power_iters"])
    YA = om.as_sparse(host["G_XA"]) @ wh["W"]
    YB = om.as_sparse(host["G_XB"]) @ wh["W_B"]
    YC = om.as_sparse(host["G_XC"]) @ wh["W_C"]
    yb = (YA.mean(axis=0), YB.mean(axis=0), YC.mean(axis=0))
    t1 = time.perf_counter()
    V, _ = ostgd.sgd_run(host["V0"], YA, YB, YC, yb, host["perm"], cfg["b"], cfg["beta0"],
                         cfg["theta"], cfg["alpha0"], max_steps=sgd_steps)
    t2 = time.perf_counter()
    opost.unwhiten(V, wh["Wplus"], cfg["theta"], False)
    ocomm.membership(YA, V, cfg["theta"])
    t3 = time.perf_counter()
    return t1 - t0, (t2 - t1) / sgd_steps, t3 - t2


def cpu_value(cfg, host, sgd_steps=10):
    pre, per_step, post = oracle_sample(cfg, host, sgd_steps)
    _, nsteps = sgd_flops(cfg)
    full = pre + nsteps * per_step + post
    samples = cfg["n_per"] * cfg["epochs"]
    sample = (f"oracle (FP64 NumPy) on the same workload: whitening+projection once "
              f"({pre:.2f} s), {sgd_steps} of the {nsteps} STGD steps ({per_step * 1e3:.1f} ms "
              f"each), unwhitening + membership ({post:.2f} s); value = {samples} samples / "
              f"(pre + {nsteps} x step + post) = {full:.2f} s")
    return samples / full, sample


def cpu_baseline(cfg, host):
    v, sample = cpu_value(cfg, host)
    return {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": sample}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cfg = dict(CFG)
    host = make_inputs(cfg, 0)
    for _ in range(args.warmup):
        cpu_value(cfg, host, sgd_steps=2)
    vals, samples_desc = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, samples_desc = cpu_value(cfg, host, sgd_steps=2)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": cfg["workload"], "nodes_per_part": cfg["n_per"],
                       "k": cfg["k"], "minibatch": cfg["b"], "epochs": cfg["epochs"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(),
                             "kind": "oracle", "sample": samples_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------
# Batched form: many independent decompositions in one persistent launch
# ----------------------------------------------------------------------------
BATCHED = dict(ks=(16, 32, 64, 128, 256), b_exp=(6, 12), pool=4, epochs=8, sigma=1e-2, beta0=5e-3,
               theta=1.0, seed=0)
def _measured_peaks():
    """HBM copy bandwidth (GB/s) and BF16 GEMM throughput (TFLOP/s) measured on
    the GB300s (MEASURED_PEAKS.json beside this file), else the values
    it held when this file was written."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 6789.0, 1888.6


HBM_PEAK_GBS, BF16_PEAK_TFLOPS = _measured_peaks()


B2T = dict(problems=16, ks=(16, 32), b_exp=(6, 12), pool_per_k=256, restarts=8,
           ladder=(8, 32, 128, 256), beta0=5e-3, sigma=1e-2, seed=7, polish_steps=5000,
           polish_beta=1e-2, polish_tol=1e-9)


def batched_time_to_target(otm, torch, dev):
    """Time to 1e-3 for the batched form against the plain FP32 kernel looped over
    the same chains, on a subset the FP64 oracle can polish: orthogonal-tensor
    problems (k in {16, 32}, b = 2^U{6..12}, n = max(4 b, 256 k) samples, sigma =
    1e-2, w ~ Dir(1), alpha0 = 0; problems with a component that drew no sample
    are redrawn), 8 Haar-random restarts each, beta_t = beta0/sqrt(t).  Reference
    per problem: the closed-form decomposition polished by full-batch FP64
    gradient steps on the explicit whitened tensor (the oracle on the CPU) until
    the gradient is below polish_tol relative to V.  Error of a problem = the
    best restart's relative reconstruction error.  Batched arm: one BF16
    persistent launch of all chains per ladder length E (timed with CUDA
    events); looped arm: each chain's FP32 run (per-epoch snapshots), its time
    per epoch x E summed over the chains.  Each arm runs twice: from the 8 Haar
    restarts (the paper's method), and with restart 0 replaced by the warm start
    (the canonical frame of the sketch T(I, I, theta_1) of the problem's samples,
    scaled by T(u, u, u)^(1/3); its time, summed over the problems, is added to
    both warm arms; the looped warm arm runs that one chain per problem)."""
    from oracle import stgd as ostgd
    c = dict(B2T)
    g = np.random.default_rng(c["seed"])
    emax = max(c["ladder"])
    probs, warm_ms = [], 0.0
    while len(probs) < c["problems"]:
        k = int(g.choice(c["ks"]))
        b = 2 ** int(g.integers(c["b_exp"][0], c["b_exp"][1] + 1))
        n = max(4 * b, c["pool_per_k"] * k)
        o = synth.orthogonal_samples(int(g.integers(1 << 30)), k, n, c["sigma"])
        cnt = np.bincount(o["h"], minlength=k)
        if (cnt == 0).any():
            continue
        Y64 = o["Y"].astype(np.float64)
        yb = Y64.mean(axis=0)
        T = ostgd.whitened_tensor_chunked(Y64, Y64, Y64, (yb, yb, yb), 0.0)

        def gfull(V):
            return V @ (V.T @ V) ** 2 - ostgd.contract_all(T, V)
        V64 = o["U"] * ((cnt / n) * o["w"] ** -1.5) ** (1.0 / 3.0)
        beta, steps = c["polish_beta"], 0
        gn = np.linalg.norm(gfull(V64)) / np.linalg.norm(V64)
        while steps < c["polish_steps"] and gn > c["polish_tol"]:
            Vn = V64 - beta * gfull(V64)
            gnn = np.linalg.norm(gfull(Vn)) / np.linalg.norm(Vn)
            if not np.isfinite(gnn) or gnn > 2 * gn:
                beta *= 0.5
                continue
            V64, gn, steps = Vn, gnn, steps + 1
        if gn > c["polish_tol"]:
            continue
        nr = np.linalg.norm(V64, axis=0)
        Y = torch.from_numpy(o["Y"]).to(dev)
        Yq, sc = otm.quantize_samples(Y, otm.PREC_BF16)
        V0 = np.stack([synth.haar_orthonormal(int(g.integers(1 << 30)), k).T
                       for _ in range(c["restarts"])])
        th = torch.from_numpy(synth.unit_vectors(int(g.integers(1 << 30)), 4, k)).to(dev)
        a0 = torch.zeros(1, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Sk, _ = otm.ws_sketch(Y[None], a0, th)
        Ef, _, _ = otm.ws_canonicalize(Sk)
        Vf = otm.ws_init_components(Ef, Y[None], a0, 1.0)[0].contiguous()
        e1.record()
        torch.cuda.synchronize()
        warm_ms += e0.elapsed_time(e1)
        probs.append({"k": k, "b": b, "n": n, "Y": Y, "Yq": Yq, "scales": sc, "Vf": Vf,
                      "ybar3": torch.from_numpy(np.stack([yb] * 3)).to(dev),
                      "perm": torch.from_numpy(synth.epoch_permutations(
                          int(g.integers(1 << 30)), n, emax)).to(dev),
                      "V0": torch.from_numpy(np.ascontiguousarray(V0, dtype=np.float32)).to(dev),
                      "lam": torch.from_numpy(nr ** 3).to(dev),
                      "U": torch.from_numpy((V64 / nr).T.copy()).to(dev),
                      "polish_steps": steps})

    def err(V, p):
        e = float(otm.recon_error(V.contiguous(), p["U"], p["lam"], 1.0)[0])
        return e if np.isfinite(e) else np.inf
    # looped plain FP32 kernel: per-epoch errors and time per epoch of every chain
    def looped(starts):
        errs = np.full((len(probs), emax), np.inf)
        epoch_ms = 0.0
        for i, p in enumerate(probs):
            spe = -(-p["n"] // p["b"])
            for V0 in starts(p):
                V = V0.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                sn = otm.sgd_run(V, p["Y"], p["Y"], p["Y"], p["ybar3"], p["perm"], emax, p["b"],
                                 c["beta0"], 1.0, 0.0, snapshot_every=spe)
                e1.record()
                torch.cuda.synchronize()
                epoch_ms += e0.elapsed_time(e1) / emax
                for E in c["ladder"]:
                    errs[i, E - 1] = min(errs[i, E - 1], err(sn[E - 1], p))
        return errs, epoch_ms
    loop_err, loop_epoch_ms = looped(lambda p: [p["V0"][r] for r in range(c["restarts"])])
    wloop_err, wloop_epoch_ms = looped(lambda p: [p["Vf"]])

    def v0(p, warm):
        V = p["V0"].clone()
        if warm:
            V[0].copy_(p["Vf"])
        return V
    ladder = []
    for E in c["ladder"]:
        row = {"epochs": E}
        for arm, warm in (("batched_bf16", False), ("batched_bf16_warm", True)):
            items = [{"Yq": p["Yq"], "scales": p["scales"], "ybar3": p["ybar3"],
                      "perm": p["perm"][:E].contiguous(), "V": v0(p, warm), "epochs": E,
                      "b": p["b"], "beta0": c["beta0"], "theta": 1.0, "alpha0": 0.0}
                     for p in probs]
            batch = otm.SgdBatch(items, otm.PREC_BF16)
            batch.launch()            # warm-up run (the chains restart below)
            batch.check()
            for it, p in zip(items, probs):
                it["V"].copy_(v0(p, warm))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.launch()
            e1.record()
            batch.check()
            berr = np.array([min(err(it["V"][r], p) for r in range(c["restarts"]))
                             for it, p in zip(items, probs)])
            row[arm] = {"ms": e0.elapsed_time(e1) + (warm_ms if warm else 0.0),
                        "median_error": float(np.median(berr)),
                        "solved": {f"{t:g}": float(np.mean(berr <= t)) for t in (1e-3, 1e-2, 1e-1)}}
        for arm, errs, ems, extra in (("looped_fp32", loop_err, loop_epoch_ms, 0.0),
                                      ("looped_fp32_warm", wloop_err, wloop_epoch_ms, warm_ms)):
            le = errs[:, E - 1]
            row[arm] = {"ms": ems * E + extra, "median_error": float(np.median(le)),
                        "solved": {f"{t:g}": float(np.mean(le <= t)) for t in (1e-3, 1e-2, 1e-1)}}
        ladder.append(row)

    def first(arm, tol, frac):
        for row in ladder:
            if row[arm]["solved"][tol] >= frac:
                return row[arm]["ms"] / 1e3
        return None
    arms = ("batched_bf16", "batched_bf16_warm", "looped_fp32", "looped_fp32_warm")
    return {"problems": (f"{len(probs)} orthogonal-tensor problems, k in {list(c['ks'])}, "
                         f"b = 2^U{{{c['b_exp'][0]}..{c['b_exp'][1]}}}, n = max(4 b, "
                         f"{c['pool_per_k']} k), sigma = {c['sigma']}, w ~ Dir(1), "
                         f"{c['restarts']} Haar restarts, beta_t = {c['beta0']:g}/sqrt(t)"),
            "reference": ("closed form polished by full-batch FP64 gradient steps on the "
                          "explicit whitened tensor (oracle, CPU) to a gradient below "
                          f"{c['polish_tol']:g}; steps per problem "
                          f"{[p['polish_steps'] for p in probs]}"),
            "chains": len(probs) * c["restarts"], "warm_start_ms": warm_ms, "ladder": ladder,
            # seconds until half of the problems (the median problem) / all of them
            # are within the tolerance, per arm; null = not within the ladder
            "seconds_to_tolerance": {
                f"{t:g}": {a: {"half": first(a, f"{t:g}", 0.5), "all": first(a, f"{t:g}", 1.0)}
                           for a in arms} for t in (1e-3, 1e-2, 1e-1)}}


def run_batched(args):
    """Whitened orthogonal-tensor problems (y = w_h^{-1/2} u_h + sigma eps, alpha0 = 0),
    k ~ U{16, 32, 64, 128, 256}, b = 2^U{6..12}, a pool of 4 b samples per problem,
    8 epochs, `restarts` Haar-random starts each; all chains in one persistent
    BF16 tensor-core launch per group (k <= 128, the restarts of a problem with
    k <= 64 stacked into one chain; k = 256 with 4- to 16-CTA clusters), captured in
    a CUDA graph.  Algorithmic flops per step of one chain (symmetric views, counted
    per restart whether stacked or not): 2 k^2 b (A = Y V) + 2 k^2 b (Y^T B) + 4 k^3
    (Gram).
    The plain FP32 kernel, looped chain by chain, is timed on the first restart of
    the first problems with k <= 128 (its limit) and extrapolated per sample."""
    import torch
    from paper_1309_0787_gb300 import otm
    dev = torch.device("cuda", 0)
    c = dict(BATCHED)
    g = np.random.default_rng(c["seed"])
    probs, flops, samples, chains = [], 0, 0, 0
    for p in range(args.problems):
        k = int(g.choice(c["ks"]))
        b = 2 ** int(g.integers(c["b_exp"][0], c["b_exp"][1] + 1))
        n = c["pool"] * b
        o = synth.orthogonal_samples(c["seed"] + 100 + p, k, n, c["sigma"])
        Y = torch.from_numpy(o["Y"]).to(dev)
        Yq, sc = otm.quantize_samples(Y, otm.PREC_BF16)
        yb = Y.double().mean(0)
        V0 = np.stack([synth.haar_orthonormal(c["seed"] + 10000 + 16 * p + r, k).T
                       for r in range(args.restarts)])
        probs.append({"Y": Y, "Yq": Yq, "scales": sc, "ybar3": torch.stack([yb] * 3).contiguous(),
                      "perm": torch.from_numpy(synth.epoch_permutations(c["seed"] + 50000 + p, n,
                                                                        c["epochs"])).to(dev),
                      "V0": torch.from_numpy(np.ascontiguousarray(V0)).to(dev),
                      "V": torch.from_numpy(np.ascontiguousarray(V0)).to(dev),
                      "epochs": c["epochs"], "b": b, "beta0": c["beta0"], "theta": c["theta"],
                      "alpha0": 0.0, "k": k, "n": n})
        steps = (n // b) * c["epochs"]
        flops += args.restarts * steps * (4 * k * k * b + 4 * k ** 3)
        samples += args.restarts * steps * b
        chains += args.restarts
    batch = otm.SgdBatch(probs, otm.PREC_BF16, cluster=args.cluster)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.launch()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    batch.check()
    sampler = ClockSampler(0)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = otm.launch_count()
    for e0, e1 in ev:
        e0.record()
        graph.replay()
        e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    batch.check()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t = statistics.mean(ms) / 1e3
    # the plain FP32 kernel looped over chains (first restart of the first problems)
    loop_probs = [p for p in probs if p["k"] <= 128][:8]   # the FP32 kernel stops at k = 128
    nloop = len(loop_probs)
    lsamples, lt = 0, 0.0
    for p in loop_probs:
        V = p["V0"][0].contiguous()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        otm.sgd_run(V, p["Y"], p["Y"], p["Y"], p["ybar3"], p["perm"], p["epochs"], p["b"],
                    p["beta0"], p["theta"], p["alpha0"])
        e1.record()
        torch.cuda.synchronize()
        lt += e0.elapsed_time(e1) / 1e3
        lsamples += (p["n"] // p["b"]) * p["epochs"] * p["b"]
    achieved = flops / t / 1e12
    return {"metric": "batched STGD throughput (samples/s), BF16 tensor cores, one persistent launch",
            "value": samples / t, "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"batched_{args.problems}x{args.restarts}_orthogonal",
                       "problems": args.problems, "restarts": args.restarts, "chains": chains,
                       "k_choices": list(c["ks"]), "minibatch": "2^U{6..12}",
                       "launches_per_step": 1 + (batch.plan.nitems_wide > 0),
                       "pool": "4 b samples", "epochs": c["epochs"], "cluster": batch.cluster,
                       "l2": "inputs larger than L2" if samples > 0 else None,
                       "chains_k256": int(batch.plan.nitems_wide),
                       "cluster_k256": int(batch.plan.cluster_wide)},
            "roofline": {"kernel": "sgd_tc_batched_kernel", "bound": "tensor",
                         "achieved": achieved, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / BF16_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)",
                         "algorithmic_flops_per_launch": flops},
            "vs_plain_fp32_loop": {"samples_per_s": lsamples / lt, "chains_timed": nloop,
                                   "speedup": (samples / t) / (lsamples / lt)},
            "time_to_1e-3": (batched_time_to_target(otm, torch, dev)
                             if not args.no_time_to_target else None),
            # one persistent kernel per graph replay (graph replays bypass the library's
            # host-side launch counter)
            "gpu_launches": args.steps * (1 + (batch.plan.nitems_wide > 0)),
            "clocks": clocks}


# ----------------------------------------------------------------------------
# Learned warm start: time to 1e-3 reconstruction error on held-out instances
# ----------------------------------------------------------------------------
WARM = dict(k=64, J=4, width=512, n_train=2000, ntr=32768, batch=256, train_epochs=2,
            lr=3e-4, n_test=8192, nte=16, beta0=0.02, epochs=300, ref_steps=3000,
            bf16_epochs=100, seed=0)


def run_warmstart(args):
    """Exact-mixture LDA instances in whitened coordinates (alpha0 ~ U[0.5, 2]).  The
    network (canonical frame of the first sketch + MLP started at the identity) is
    trained on `ntr` generated instances; on `nte` held-out instances full-batch
    STGD (b = n, beta_t = beta0/sqrt(t)) runs from (a) a Haar-random start, FP32
    (the paper's method), (b) the learned start, FP32, (c) the learned start,
    BF16 tensor cores, (d) the learned start, BF16 for `bf16_epochs` then FP32.
    Error after every epoch = relative reconstruction error against a reference:
    `ref_steps` FP32 full-batch steps from the learned start.  Reported per method:
    fraction of instances reaching 1e-3 within `epochs`, median epochs and median
    seconds (epochs x measured step time)."""
    import torch
    from paper_1309_0787_gb300 import otm
    c = dict(WARM)
    if args.k:
        c["k"] = args.k
    k, J, h = c["k"], c["J"], c["width"]
    din, dout = J * k * k, k * k
    dev = torch.device("cuda", 0)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    inst = synth.whitened_lda_instances(c["seed"], c["ntr"] + c["nte"], k)
    th = torch.from_numpy(synth.unit_vectors(c["seed"] + 1, J, k)).to(dev)
    m = torch.from_numpy(inst["m"]).to(dev)
    al = torch.from_numpy(inst["alpha32"]).to(dev)
    a0 = torch.from_numpy(inst["alpha0"]).to(dev)
    Us = torch.from_numpy(inst["U"].astype(np.float32)).to(dev)
    lam = torch.from_numpy(inst["lam"].astype(np.float32)).to(dev)
    # training data: generate, sketch, canonical frame (in chunks)
    X = torch.empty(c["ntr"], din, dtype=torch.bfloat16, device=dev)
    E = torch.empty(c["ntr"], k, k, dtype=torch.float32, device=dev)
    e0, e1 = ev(), ev()
    e0.record()
    for c0 in range(0, c["ntr"], 512):
        c1 = min(c0 + 512, c["ntr"])
        Y = otm.ws_generate(m[c0:c1].contiguous(), al[c0:c1].contiguous(), c["n_train"],
                            c["seed"] + 2, first=c0)
        S, _ = otm.ws_sketch(Y, a0[c0:c1].contiguous(), th)
        Ec, _, Xc = otm.ws_canonicalize(S)
        X[c0:c1] = Xc
        E[c0:c1] = Ec
    e1.record()
    torch.cuda.synchronize()
    gen_ms = e0.elapsed_time(e1)
    Ut = otm.ws_rotate(E, Us[:c["ntr"]].contiguous(), transpose=True)
    # network, started at the canonical frame (b3 = vec(I), W3 small)
    g = np.random.default_rng(c["seed"] + 3)
    W1 = g.standard_normal((h, din)) / np.sqrt(din)
    W2 = g.standard_normal((h, h)) / np.sqrt(h)
    W3 = 0.01 * g.standard_normal((dout, h)) / np.sqrt(h)
    params = np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), W3.ravel(),
                             np.eye(k).ravel()]).astype(np.float32)
    net = otm.Mlp(din, h, dout, params)
    B = c["batch"]
    steps = c["train_epochs"] * c["ntr"] // B
    losses = []
    e0.record()
    for st in range(steps):
        i0 = (st * B) % c["ntr"]
        l = net.train_step(X[i0:i0 + B], Ut[i0:i0 + B], lam[i0:i0 + B], k, c["lr"])
        if st % max(1, steps // 8) == 0 or st == steps - 1:
            losses.append(l)
    e1.record()
    torch.cuda.synchronize()
    net.check(B)
    train_ms = e0.elapsed_time(e1)
    losses = [round(float(x.mean()), 4) for x in losses]
    # held-out instances
    nte, n = c["nte"], c["n_test"]
    lo = c["ntr"]
    Yt = otm.ws_generate(m[lo:].contiguous(), al[lo:].contiguous(), n, c["seed"] + 4, first=lo)
    St, _ = otm.ws_sketch(Yt, a0[lo:].contiguous(), th)
    Et, _, Xt = otm.ws_canonicalize(St)
    nb = ((nte + 7) // 8) * 8
    Xpad = torch.zeros(nb, din, dtype=torch.bfloat16, device=dev)
    Xpad[:nte] = Xt
    U0 = otm.ws_rotate(Et, net.infer(Xpad, k)[:nte].contiguous())
    Vwarm = otm.ws_init_components(U0, Yt, a0[lo:].contiguous(), 1.0)
    held = {"network": -float(otm.ws_loss_grad(U0, Us[lo:].contiguous(),
                                                lam[lo:].contiguous())[0].mean()),
            "frame": -float(otm.ws_loss_grad(Et, Us[lo:].contiguous(),
                                              lam[lo:].contiguous())[0].mean())}
    kappa = 1.0
    results = {nm: {"epochs": [], "reached": 0} for nm in
               ("fp32_random", "fp32_warm", "bf16_warm", "bf16_then_fp32_warm")}
    tstep = {nm: [] for nm in results}
    for i in range(nte):
        Y = Yt[i].contiguous()
        yb = torch.stack([Y.double().mean(0)] * 3).contiguous()
        q = otm.quantize_samples(Y, otm.PREC_BF16)
        Vw = Vwarm[i].contiguous()
        Vref = Vw.clone()
        otm.sgd_run(Vref, Y, Y, Y, yb, None, c["ref_steps"], n, c["beta0"], 1.0, float(a0[lo + i]))
        nr = Vref.double().norm(dim=1)
        lam_r = (kappa * nr ** 3).contiguous()
        U_r = (Vref.double() / nr[:, None]).contiguous()

        def errs(snaps):
            return [float(otm.recon_error(snaps[j].contiguous(), U_r, lam_r, 1.0)[0])
                    for j in range(snaps.shape[0])]

        def timed(fn):
            t0, t1 = ev(), ev()
            t0.record()
            out = fn()
            t1.record()
            torch.cuda.synchronize()
            return out, t0.elapsed_time(t1)

        a0i = float(a0[lo + i])
        Vr = torch.from_numpy(synth.haar_orthonormal(c["seed"] + 500 + i, k).T.copy()).to(dev)
        runs = {}
        runs["fp32_random"] = timed(lambda: otm.sgd_run(Vr, Y, Y, Y, yb, None, c["epochs"], n,
                                                        c["beta0"], 1.0, a0i, snapshot_every=1))
        V1 = Vw.clone()
        runs["fp32_warm"] = timed(lambda: otm.sgd_run(V1, Y, Y, Y, yb, None, c["epochs"], n,
                                                      c["beta0"], 1.0, a0i, snapshot_every=1))
        V2 = Vw.clone()
        runs["bf16_warm"] = timed(lambda: otm.sgd_run_lp(V2, q, q, q, yb, None, c["epochs"], n,
                                                         c["beta0"], 1.0, a0i, otm.PREC_BF16,
                                                         snapshot_every=1))
        for nm, (snaps, ms) in runs.items():
            tstep[nm].append(ms / c["epochs"])
            e = errs(snaps)
            hit = next((j for j, x in enumerate(e) if x <= 1e-3), None)
            if hit is not None:
                results[nm]["reached"] += 1
                results[nm]["epochs"].append(hit + 1)
        # mixed: BF16 epochs, then FP32 from the BF16 iterate
        V3 = Vw.clone()
        s16, _ = timed(lambda: otm.sgd_run_lp(V3, q, q, q, yb, None, c["bf16_epochs"], n,
                                              c["beta0"], 1.0, a0i, otm.PREC_BF16,
                                              snapshot_every=1))
        s32, _ = timed(lambda: otm.sgd_run(V3, Y, Y, Y, yb, None, c["epochs"] - c["bf16_epochs"],
                                           n, c["beta0"], 1.0, a0i, snapshot_every=1))
        e = errs(s16) + errs(s32)
        hit = next((j for j, x in enumerate(e) if x <= 1e-3), None)
        tstep["bf16_then_fp32_warm"].append(0.0)
        if hit is not None:
            results["bf16_then_fp32_warm"]["reached"] += 1
            results["bf16_then_fp32_warm"]["epochs"].append(hit + 1)
    t32 = statistics.median(tstep["fp32_warm"])
    t16 = statistics.median(tstep["bf16_warm"])
    out = {}
    for nm, r in results.items():
        med = statistics.median(r["epochs"]) if r["epochs"] else None
        if nm == "bf16_then_fp32_warm":
            sec = None if med is None else (min(med, c["bf16_epochs"]) * t16 +
                                            max(0, med - c["bf16_epochs"]) * t32) / 1e3
        else:
            sec = None if med is None else med * statistics.median(tstep[nm]) / 1e3
        out[nm] = {"reached_1e-3": f"{r['reached']}/{nte}", "median_epochs": med,
                   "median_seconds": sec,
                   "step_ms": statistics.median(tstep[nm]) if tstep[nm][0] else None}
    plain = out["fp32_random"]["median_seconds"]
    best = min([v["median_seconds"] for nm, v in out.items()
                if nm != "fp32_random" and v["median_seconds"] is not None], default=None)
    return {"metric": "time to 1e-3 reconstruction error: warm-started vs plain FP32 STGD",
            "value": best, "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "steps": 1, "warmup": 0, "dtype": "bf16+f32", "data": "synthetic",
            "vs_baseline": None,
            "config": {"workload": f"warmstart_lda_whitened_k{k}", "k": k, "J": J,
                       "width": h, "train_instances": c["ntr"],
                       "train_samples_per_instance": c["n_train"], "heldout": nte,
                       "samples_per_heldout": n, "minibatch": "full (b = n)",
                       "beta0": c["beta0"], "epochs": c["epochs"],
                       "reference": f"{c['ref_steps']} FP32 full-batch steps from the learned start"},
            "plain_fp32_random_init": out["fp32_random"], "methods": out,
            "plain_reached_at_all": plain is not None,
            "heldout_T_captured": held, "train_loss_trace": losses,
            "generate_sketch_ms_per_instance": gen_ms / c["ntr"],
            "train_instances_per_s": steps * B / (train_ms / 1e3)}


# ----------------------------------------------------------------------------
def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


WHITEN = dict(workload="lda_30000x20000_k50_whitening", n_docs=30000, d=20000, k=50,
              alpha_i=0.01, word_conc=0.05, doc_len=300, oversample=20, power_iters=2, seed=0)


def run_whitening(args):
    """Randomised whitening of a topic model's M2, both forms, on one LDA corpus
    (30,000 documents of Poisson(300) words over 20,000 words, k = 50,
    alpha0 = 0.5): the range finder (Gaussian S, k + 20 columns, 2 power
    iterations, tall-thin QR) and the paper's Nystrom form (Algorithm 2,
    signed column selection, k~ = 2k).  Per form: device time per call (median
    of `steps`, L2 flushed before each; each call ends with its host-checked
    eigenvalue flag) and the whitening deviation max |W^T M2 W - I| with M2
    applied implicitly."""
    import torch
    from paper_1309_0787_gb300 import otm
    c = dict(WHITEN)
    dev = torch.device("cuda", 0)
    k, d = c["k"], c["d"]
    alpha0 = k * c["alpha_i"]
    corpus = synth.lda_corpus(c["seed"], c["n_docs"], d, k, c["alpha_i"], c["word_conc"],
                              c["doc_len"], poisson_len=True)
    Xd = otm.DeviceCSR.from_host(corpus["X"], dev)
    S_rf = torch.from_numpy(synth.gaussian(c["seed"] + 1, d, k + c["oversample"])).to(dev)
    S_ny = torch.from_numpy(synth.signed_column_selection(c["seed"] + 2, d, 2 * k)).to(dev)
    forms = {"range_finder": lambda: otm.whiten_topic(Xd, S_rf, k, c["power_iters"], alpha0),
             "nystrom": lambda: otm.whiten_topic_nystrom(Xd, S_ny, k, alpha0)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mom = otm.topic_moments(Xd)
    sampler = ClockSampler(0)
    sampler.start()
    res = {}
    for name, f in forms.items():
        for _ in range(args.warmup):
            f()
        ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = f()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        W = out["W"]
        MW = otm.topic_m2_apply(Xd, mom, alpha0, W)
        dev_max = (W.double().t() @ MW.double() - torch.eye(k, dtype=torch.float64, device=dev))
        res[name] = {"ms": statistics.median(ms), "ms_all": ms,
                     "whitening_deviation_max": float(dev_max.abs().max()),
                     "columns": int(out["Q"].shape[1])}
    clocks = sampler.stop()
    return {"metric": "randomised whitening time (ms), Nystrom form (Algorithm 2)",
            "value": res["nystrom"]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["nystrom"]["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": c["workload"], "docs": c["n_docs"], "vocabulary": d, "k": k,
                       "alpha0": alpha0, "nnz": int(corpus["X"].nnz),
                       "l2": "flushed before each call (256 MiB write)"},
            "forms": res, "clocks": clocks,
            "note": ("the range finder satisfies W^T M2 W = I by construction (Rayleigh-Ritz on "
                     "its basis), so its deviation is float32 rounding; the Nystrom form's "
                     "deviation measures how much of M2 its column selection misses")}


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sym_sgd_flops(n, b, k, epochs):
    """Algorithmic flops of an STGD run with symmetric views: per step
    2k^2 b_s (A = V^T Y) + 2k^2 b_s (Y^T B^T) + 4k^3 (Gram term)."""
    sizes = [min(b, n - s) for s in range(0, n, b)] * epochs
    return sum(4 * k * k * bs + 4 * k ** 3 for bs in sizes)


# ----------------------------------------------------------------------------
# The default line: the whole hot path on a large synthetic LDA corpus
# ----------------------------------------------------------------------------
LDA = dict(workload="lda_300000x100000_k100_b1024_fp32", n_docs=300000, d=100000, k=100,
           alpha_i=0.01, word_conc=0.05, doc_len=300, oversample=20, power_iters=2, b=1024,
           epochs=20, beta0=1e-2, theta=1.0, seed=0, check_docs=256)


def lda_corpus_cached(c, seed):
    """The synthetic corpus (about 17 s to draw on one core), cached as an .npz in
    the system temp directory so that a second process on the same machine (the
    reference arm) loads it instead.  The cache holds only what synth drew."""
    import tempfile
    key = (f"otm_lda_{c['n_docs']}x{c['d']}_k{c['k']}_a{c['alpha_i']}_w{c['word_conc']}"
           f"_l{c['doc_len']}_s{seed}.npz")
    path = os.path.join(tempfile.gettempdir(), "otm_bench_cache", key)
    if os.path.exists(path):
        try:
            z = np.load(path)
            X = synth.CSR(z["row_ptr"], z["col"], z["val"], tuple(int(v) for v in z["shape"]))
            return {"X": X, "mu": z["mu"], "cached": True}
        except Exception:
            pass
    corpus = synth.lda_corpus(seed, c["n_docs"], c["d"], c["k"], c["alpha_i"], c["word_conc"],
                              c["doc_len"], poisson_len=True, zipf=True)
    X = corpus["X"]
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, row_ptr=X.row_ptr, col=X.col, val=X.val, shape=np.array(X.shape),
                 mu=corpus["mu"])
        os.replace(tmp, path)
    except OSError:
        pass
    return {"X": X, "mu": corpus["mu"], "cached": False}


def lda_inputs(c, rank=0):
    """Seeded inputs of one decomposition (rank r draws seed + 1000 r): the corpus,
    the range finder's Gaussian projection S (d x (k + oversample)), the epoch
    permutations and a Haar-random start V0 (columns = components)."""
    s = c["seed"] + 1000 * rank
    t0 = time.perf_counter()
    corpus = lda_corpus_cached(c, s)
    gen_s = time.perf_counter() - t0
    d, k = c["d"], c["k"]
    n = corpus["X"].shape[0]
    return {"X": corpus["X"], "mu": corpus["mu"], "gen_s": gen_s, "cached": corpus["cached"],
            "S": synth.gaussian(s + 1, d, k + c["oversample"]),
            "perm": synth.epoch_permutations(s + 3, n, c["epochs"]),
            "V0": synth.haar_orthonormal(s + 4, k)}


class LdaPath:
    """The hot path on the GPU: topic-model whitening (range finder) ->
    projection -> means -> FP32 STGD (one persistent launch) -> unwhitening."""

    def __init__(self, otm, torch, c, host, device):
        self.otm, self.torch, self.c, self.dev, self.host = otm, torch, c, device, host
        self.upload()

    def upload(self, pinned=None):
        t, otm = self.torch, self.otm
        if pinned is None:
            self.Xd = otm.DeviceCSR.from_host(self.host["X"], self.dev)
            self.S = t.from_numpy(self.host["S"]).to(self.dev)
            self.perm = t.from_numpy(self.host["perm"]).to(self.dev)
            self.V0t = t.from_numpy(self.host["V0"].T.copy()).to(self.dev)
        else:
            self.Xd = otm.DeviceCSR(*(a.to(self.dev, non_blocking=True) for a in pinned["X"]),
                                    self.host["X"].shape)
            self.S = pinned["S"].to(self.dev, non_blocking=True)
            self.perm = pinned["perm"].to(self.dev, non_blocking=True)
            self.V0t = pinned["V0t"].to(self.dev, non_blocking=True)

    def front(self):
        c, otm = self.c, self.otm
        wh = otm.whiten_topic(self.Xd, self.S, c["k"], c["power_iters"], c["k"] * c["alpha_i"])
        Y = otm.project(self.Xd, wh["W"], wh["row_invlen"])
        yb3 = self.torch.empty(3, c["k"], dtype=self.torch.float64, device=self.dev)
        otm.column_mean(Y, out=yb3[0])
        yb3[1].copy_(yb3[0])      # device-to-device copies (symmetric views)
        yb3[2].copy_(yb3[0])
        return wh, Y, yb3

    def step(self, ev=None):
        c, otm = self.c, self.otm
        if ev:
            ev["w0"].record()
        wh, Y, yb3 = self.front()
        V = self.V0t.clone()
        if ev:
            ev["s0"].record()
        otm.sgd_run(V, Y, Y, Y, yb3, self.perm, c["epochs"], c["b"], c["beta0"], c["theta"],
                    c["k"] * c["alpha_i"])
        if ev:
            ev["s1"].record()
        out = otm.unwhiten(V, wh["Q"], wh["Cp"], c["theta"], True)
        self.last = (wh, Y, yb3, V)
        return out


def lda_oracle_checks(c, X, W, Y_docs, docs, Yb, yb, V0, V1):
    """FP64 oracle checks of single stages on a sample, each fed the previous
    stage's GPU output: the projection y_t = W^T c_t / l_t of the documents
    `docs` (Section 3.1), and one STGD step (Lemma 3) on the minibatch Yb from V0
    (columns = components) for each precision's result V1 (same orientation).
    Step errors: G = (V0 - V1) / beta0 against the oracle's G64, as
    ||G - G64|| / (||kappa G_gram|| + ||G_data||) over the whole matrix and for
    the worst component, and the update relative to its own norm."""
    from oracle import moments as om
    from oracle import stgd as ostgd
    Xs = om.as_sparse(X)[docs]
    lens = np.asarray(Xs.sum(axis=1)).ravel()
    y_ref = (Xs @ np.asarray(W, dtype=np.float64)) / lens[:, None]
    Yb = np.asarray(Yb, dtype=np.float64)
    yb = np.asarray(yb, dtype=np.float64)
    V0 = np.asarray(V0, dtype=np.float64)
    a0 = c["k"] * c["alpha_i"]
    G = ostgd.grad_implicit(V0, Yb, Yb, Yb, (yb, yb, yb), c["theta"], a0)
    gram = ostgd.kappa(c["theta"]) * V0 @ (V0.T @ V0) ** 2
    den = np.linalg.norm(gram) + np.linalg.norm(gram - G)
    den_col = np.linalg.norm(gram, axis=0) + np.linalg.norm(gram - G, axis=0)
    step = {}
    for p, v in V1.items():
        Gk = (V0 - np.asarray(v, dtype=np.float64)) / c["beta0"]
        step[p] = {"grad_rel_err": float(np.linalg.norm(Gk - G) / den),
                   "grad_rel_err_worst_component":
                       float((np.linalg.norm(Gk - G, axis=0) / den_col).max()),
                   "update_rel_err": _rel(Gk, G)}
    return {"projection_rows_rel_err": _rel(Y_docs, y_ref), "step": step}


def lda_precisions(otm, torch, path, c, host, fp32_sgd_ms):
    """The precision form on the same whitened samples: sample quantisation, then
    the 20 epochs of STGD from the same start in BF16, in FP8 and in FP8 with
    two-term samples (tensor cores, FP32 accumulation; medians of three runs).  Errors: one step of each
    precision against the FP64 oracle (lda_oracle_checks), and the 20-epoch
    results against the FP32 one (relative reconstruction error of the
    components, relative error of the unwhitened topics)."""
    from oracle import post as opost
    wh, Y, yb3, V32 = path.last
    k, b, ep, th = c["k"], c["b"], c["epochs"], c["theta"]
    a0 = k * c["alpha_i"]
    n = Y.shape[0]
    dev = Y.device
    res = {"fp32": {"sgd_ms": fp32_sgd_ms, "samples_per_s": n * ep / (fp32_sgd_ms / 1e3)}}
    V = {"fp32": V32}
    precs = {"bf16": otm.PREC_BF16, "fp8": otm.PREC_FP8, "fp8x2": otm.PREC_FP8X2}
    for nm, pr in precs.items():
        tq, ts = [], []
        for _ in range(3):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            q = otm.quantize_samples(Y, pr)
            e[1].record()
            Vp = path.V0t.clone()
            otm.sgd_run_lp(Vp, q, q, q, yb3, path.perm, ep, b, c["beta0"], th, a0, pr)
            e[2].record()
            torch.cuda.synchronize()
            tq.append(e[0].elapsed_time(e[1]))
            ts.append(e[1].elapsed_time(e[2]))
        V[nm] = Vp
        res[nm] = {"quantize_ms": statistics.median(tq), "sgd_ms": statistics.median(ts),
                   "samples_per_s": n * ep / (statistics.median(ts) / 1e3)}
    nr = V32.double().norm(dim=1)
    kappa = 0.5 * (1.0 + th)
    lam = (kappa * nr ** 3).contiguous()
    U = (V32.double() / nr[:, None]).contiguous()
    topics = {nm: otm.unwhiten(v, wh["Q"], wh["Cp"], th, True)["comps"] for nm, v in V.items()}
    for nm in precs:
        res[nm]["after_run_vs_fp32"] = {
            "recon_rel_err": float(otm.recon_error(V[nm], U, lam, th)[0]),
            "topics_rel_err": float((topics[nm] - topics["fp32"]).norm() / topics["fp32"].norm())}
    # one step of each precision from the Haar start on the first minibatch
    docs = host["perm"][0][:b].astype(np.int64)
    idx = torch.from_numpy(docs).to(dev)
    Yb = Y[idx].contiguous()
    V1 = {"fp32": path.V0t.clone()}
    otm.sgd_step(V1["fp32"], Yb, Yb, Yb, yb3, th, c["beta0"], a0)
    for nm, pr in precs.items():
        qb = otm.quantize_samples(Yb, pr)
        V1[nm] = path.V0t.clone()
        otm.sgd_run_lp(V1[nm], qb, qb, qb, yb3, None, 1, b, c["beta0"], th, a0, pr)
    torch.cuda.synchronize()
    cd = docs[: c["check_docs"]]
    checks = lda_oracle_checks(c, host["X"], wh["W"].cpu().numpy(), Y[idx[: c["check_docs"]]]
                               .cpu().numpy(), cd, Yb.cpu().numpy(), yb3[0].cpu().numpy(),
                               host["V0"], {nm: v.cpu().numpy().T for nm, v in V1.items()})
    for nm in res:
        res[nm]["one_step_vs_fp64_oracle"] = checks["step"][nm]
    Qh = wh["Q"].cpu().numpy().astype(np.float64)
    mu_ref = opost.unwhiten(V32.cpu().numpy().T.astype(np.float64),
                            Qh @ wh["Cp"].cpu().numpy(), th, True)["mu"]
    res["stage_checks_vs_fp64_oracle"] = {
        "projection_rows_rel_err": checks["projection_rows_rel_err"],
        "unwhiten_rel_err": _rel(topics["fp32"].cpu().numpy(), mu_ref),
        "sample": f"projection of {len(cd)} documents; one STGD step on the first minibatch "
                  f"({b} documents) from the Haar start; unwhitening of the FP32 result"}
    return res


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def lda_oracle_sample(c, host, fracs, stgd_steps, project_frac=1.0):
    """Times the oracle (FP64 NumPy/SciPy) on the host cores, on the line's inputs:
      whitening (range finder, Section 4.2) of the first f n documents for each f
      in `fracs`; its full-corpus time by a linear fit in f (a dense part that
      does not depend on the documents plus a part proportional to them);
      projection and means (Section 3.1) of the first project_frac n documents,
      scaled to all of them;
      `stgd_steps` steps of the matrix-form implicit STGD (Lemma 3) with the
      line's schedule (None: the whole schedule, run to completion);
      unwhitening (Lemma 4).
    Returns the seconds of each part, for the whole workload."""
    from oracle import moments as om
    from oracle import post as opost
    from oracle import stgd as ostgd
    from oracle import whiten as ow
    X = host["X"]
    n = X.shape[0]
    k, a0 = c["k"], c["k"] * c["alpha_i"]
    S = host["S"].astype(np.float64)
    t_wh, wh, passed = [], None, []
    for f in fracs:
        Xf = X.row_slice(0, max(1, int(round(f * n))))
        t0 = time.perf_counter()
        try:
            wh = ow.range_finder_whiten(lambda Z, Xf=Xf: om.topic_second_moment_apply(Xf, Z, a0),
                                        S, k, c["power_iters"])
            passed.append(True)
        except ow.NotPositiveDefinite:
            # a small share of the documents may leave fewer than k positive
            # eigenvalues; the check is the whitening's last step, so the time
            # is that of the whole whitening
            passed.append(False)
        t_wh.append(time.perf_counter() - t0)
    if wh is None:   # stand-ins of the same shapes for the timing of the later stages
        wh = {"W": S[:, :k].copy(), "Wplus": S[:, :k].copy()}
    if len(fracs) > 1:
        slope = (t_wh[-1] - t_wh[0]) / (fracs[-1] - fracs[0])
        whiten_s = max(t_wh[-1] + slope * (1.0 - fracs[-1]), t_wh[-1])
    else:
        whiten_s = t_wh[0] / fracs[0]
    npj = max(1, int(round(project_frac * n)))
    t0 = time.perf_counter()
    Xs = om.as_sparse(X.row_slice(0, npj))
    Y = (Xs @ wh["W"]) / om.doc_lengths(Xs)[:, None]
    yb = Y.mean(axis=0)
    project_s = (time.perf_counter() - t0) * n / npj
    if npj < n:   # the STGD reads every document: tile the projected rows
        Y = np.resize(Y, (n, k))
    total = ostgd.steps_per_epoch(n, c["b"]) * c["epochs"]
    steps = total if stgd_steps is None else min(stgd_steps, total)
    t0 = time.perf_counter()
    V, _ = ostgd.sgd_run(host["V0"].astype(np.float64), Y, Y, Y, (yb, yb, yb), host["perm"],
                         c["b"], c["beta0"], c["theta"], a0, max_steps=steps, gemm=True)
    stgd_s = (time.perf_counter() - t0) * total / steps
    t0 = time.perf_counter()
    opost.unwhiten(V, wh["Wplus"], c["theta"], True)
    post_s = time.perf_counter() - t0
    return {"whiten_s": whiten_s, "whiten_sample_s": t_wh, "whiten_sample_positive": passed,
            "project_means_s": project_s,
            "stgd_s": stgd_s, "stgd_steps_run": steps, "stgd_steps_total": total,
            "unwhiten_s": post_s}


def lda_cpu_baseline(c, host):
    """The CPU baseline of the default line: lda_oracle_sample with the STGD run
    to completion (all 5,860 steps) and the whitening extrapolated from 5 % and
    10 % of the documents."""
    r = lda_oracle_sample(c, host, (0.05, 0.10), None)
    n = host["X"].shape[0]
    tot = r["whiten_s"] + r["project_means_s"] + r["stgd_s"] + r["unwhiten_s"]
    return {"value": n * c["epochs"] / tot, "unit": UNIT, "cores": blas_threads(),
            "kind": "oracle", "cpu": cpu_model(),
            "sample": (f"FP64 oracle on the host cores: the matrix-form implicit STGD run to "
                       f"completion ({r['stgd_steps_total']} steps, {r['stgd_s']:.1f} s); the "
                       f"range-finder whitening timed on 5 % and 10 % of the documents "
                       f"({r['whiten_sample_s'][0]:.1f} s, {r['whiten_sample_s'][1]:.1f} s) and "
                       f"extrapolated linearly to all ({r['whiten_s']:.1f} s); projection and "
                       f"means of all documents ({r['project_means_s']:.1f} s); unwhitening "
                       f"({r['unwhiten_s']:.2f} s); value = samples / total "
                       f"({tot:.1f} s)"),
            "seconds": r}


def run_lda_reference(args, rank, world):
    """The reference arm of the default line: the oracle on the host cores (rank 0
    only), every step a bounded sample of the workload: the whitening on 1 % and
    2 % of the documents (extrapolated), the projection of 2 % (scaled), 100 of
    the 5,860 STGD steps (scaled), the unwhitening."""
    if rank != 0:
        return None
    c = dict(LDA)
    host = lda_inputs(c, 0)
    n = host["X"].shape[0]

    def one():
        r = lda_oracle_sample(c, host, (0.01, 0.02), 100, project_frac=0.02)
        return r, r["whiten_s"] + r["project_means_s"] + r["stgd_s"] + r["unwhiten_s"]

    for _ in range(args.warmup):
        one()
    vals, r = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, tot = one()
        vals.append(n * c["epochs"] / tot)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    sample = (f"FP64 oracle on the host cores, per step: whitening on 1 % and 2 % of the "
              f"documents extrapolated to all ({r['whiten_s']:.1f} s), projection and means of "
              f"2 % scaled ({r['project_means_s']:.1f} s), {r['stgd_steps_run']} of the "
              f"{r['stgd_steps_total']} matrix-form STGD steps scaled ({r['stgd_s']:.1f} s), "
              f"unwhitening ({r['unwhiten_s']:.2f} s)")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": c["workload"], "docs": n, "vocabulary": c["d"],
                       "k": c["k"], "minibatch": c["b"], "epochs": c["epochs"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(),
                             "kind": "oracle", "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


T2T = dict(k=64, n=300000, b=1024, sigma=1e-2, conc=20.0, beta0=1e-3, epochs=60, J=4,
           polish_steps=4000, polish_beta=2e-2, polish_tol=1e-11, seed=0)


def time_to_target(otm, torch, dev):
    """Time to 1e-3 reconstruction error on a decomposition with a known answer,
    at the default line's sample count and minibatch: whitened samples of an
    orthogonal tensor (y = w_h^{-1/2} u_h + sigma eps, h ~ Cat(w), w ~ Dir(20 1_k),
    alpha0 = 0, so Lemma 3 reduces to the plain third moment), k = 64,
    n = 300,000, b = 1,024, sigma = 1e-2.  Its sample tensor is orthogonally
    decomposable up to O(sigma^2): components u_h, eigenvalues
    lambda_h = (n_h / n) w_h^{-3/2}.  The reference is that decomposition
    polished by full-batch FP64 gradient steps on the explicit k^3 whitened
    tensor of the samples (the FP64 oracle on the CPU); its residual is the
    oracle's implicit-form gradient over all samples.  Arms (each timed on the
    GPU, error of the epoch snapshots against the reference):
      plain_fp32  -- the paper's method: Haar-random start, FP32 STGD;
      warm_fp32   -- the warm start (sketch T(I, I, theta_1) of the samples, its
                     eigenvectors as directions, scaled by T(u, u, u)^(1/3)), then FP32 STGD;
      warm_bf16   -- the same start, BF16 tensor-core STGD.
    Time to 1e-3 = warm-start time + (first epoch whose snapshot is within 1e-3)
    x the run's time per epoch."""
    from oracle import stgd as ostgd
    c = dict(T2T)
    k, n, b, ep = c["k"], c["n"], c["b"], c["epochs"]
    spe = (n + b - 1) // b
    o = synth.orthogonal_samples(c["seed"] + 17, k, n, c["sigma"], conc=c["conc"])
    cnt = np.bincount(o["h"], minlength=k)
    lam0 = (cnt / n) * o["w"] ** -1.5
    Y = torch.from_numpy(o["Y"]).to(dev)
    yb3 = torch.from_numpy(np.stack([o["Y"].astype(np.float64).mean(axis=0)] * 3)).to(dev)
    perm = torch.from_numpy(synth.epoch_permutations(c["seed"] + 18, n, ep)).to(dev)
    # reference: the closed form, polished in FP64 on the explicit tensor (the
    # gradient kappa V (V^T V)^o2 - T(V, V, I) of Lemma 3, full batch)
    Y64 = o["Y"].astype(np.float64)
    ybh = Y64.mean(axis=0)
    T = ostgd.whitened_tensor_chunked(Y64, Y64, Y64, (ybh, ybh, ybh), 0.0)
    Vcf = o["U"] * lam0 ** (1.0 / 3.0)            # columns = components

    def grad_full(V):
        return V @ (V.T @ V) ** 2 - ostgd.contract_all(T, V)
    V64, beta, steps = Vcf.copy(), c["polish_beta"], 0
    gn = np.linalg.norm(grad_full(V64)) / np.linalg.norm(V64)
    while steps < c["polish_steps"] and gn > c["polish_tol"]:
        Vn = V64 - beta * grad_full(V64)
        gnn = np.linalg.norm(grad_full(Vn)) / np.linalg.norm(Vn)
        if not np.isfinite(gnn) or gnn > 2 * gn:
            beta *= 0.5
            continue
        V64, gn, steps = Vn, gnn, steps + 1

    def resid(V):   # the implicit-form gradient over all samples (other code path)
        G = ostgd.grad_implicit_gemm(V, Y64, Y64, Y64, (ybh, ybh, ybh), 1.0, 0.0)
        return float(np.linalg.norm(G) / np.linalg.norm(V))
    nr = np.linalg.norm(V64, axis=0)
    lam = torch.from_numpy(nr ** 3).to(dev)
    U = torch.from_numpy((V64 / nr).T.copy()).to(dev)     # row i = unit component i
    Vcf_t = torch.from_numpy(Vcf.T.astype(np.float32).copy()).to(dev)

    def run(V0, prec):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        V = V0.clone()
        q = otm.quantize_samples(Y, prec) if prec is not None else None
        torch.cuda.synchronize()
        e0.record()
        if prec is None:
            sn = otm.sgd_run(V, Y, Y, Y, yb3, perm, ep, b, c["beta0"], 1.0, 0.0,
                             snapshot_every=spe)
        else:
            sn = otm.sgd_run_lp(V, q, q, q, yb3, perm, ep, b, c["beta0"], 1.0, 0.0, prec,
                                snapshot_every=spe)
        e1.record()
        torch.cuda.synchronize()
        return sn, e0.elapsed_time(e1) / ep

    def report(sn, epoch_ms, start_ms):
        errs = [float(otm.recon_error(sn[i].contiguous(), U, lam, 1.0)[0])
                for i in range(sn.shape[0])]
        hit = next((i + 1 for i, e in enumerate(errs) if e <= 1e-3), None)
        return {"epochs_to_1e-3": hit,
                "seconds_to_1e-3": None if hit is None else (start_ms + hit * epoch_ms) / 1e3,
                "start_ms": start_ms, "epoch_ms": epoch_ms, "final_error": errs[-1],
                "error_by_epoch": [float(f"{e:.4g}") for e in errs[::3]] + [float(f"{errs[-1]:.4g}")]}

    V0h = torch.from_numpy(synth.haar_orthonormal(c["seed"] + 19, k).T.copy()).to(dev)
    out = {}
    sn, ms = run(V0h, None)
    out["plain_fp32"] = report(sn, ms, 0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    th = torch.from_numpy(synth.unit_vectors(c["seed"] + 20, c["J"], k)).to(dev)
    a0 = torch.zeros(1, dtype=torch.float64, device=dev)
    e0.record()
    S, _ = otm.ws_sketch(Y[None], a0, th)
    E, _, _ = otm.ws_canonicalize(S)
    Vw = otm.ws_init_components(E, Y[None], a0, 1.0)[0].contiguous()
    e1.record()
    torch.cuda.synchronize()
    warm_ms = e0.elapsed_time(e1)
    sn, ms = run(Vw, None)
    out["warm_fp32"] = report(sn, ms, warm_ms)
    sn, ms = run(Vw, otm.PREC_BF16)
    out["warm_bf16"] = report(sn, ms, warm_ms)
    best = min((v["seconds_to_1e-3"] for v in out.values() if v["seconds_to_1e-3"] is not None),
               default=None)
    plain = out["plain_fp32"]["seconds_to_1e-3"]
    return {"problem": (f"whitened orthogonal tensor, k = {k}, n = {n}, b = {b}, sigma = "
                        f"{c['sigma']}, w ~ Dir({c['conc']:g} 1_k), alpha0 = 0, theta = 1, "
                        f"beta_t = {c['beta0']:g}/sqrt(t), {ep} epochs, seed {c['seed']}"),
            "reference": (f"closed-form decomposition (u_h, lambda_h = (n_h/n) w_h^-1.5) "
                          f"polished by {steps} full-batch FP64 gradient steps on the explicit "
                          f"whitened tensor (oracle, CPU)"),
            "reference_grad_rel": resid(V64), "closed_form_grad_rel": resid(Vcf),
            "closed_form_vs_reference_error": float(otm.recon_error(Vcf_t, U, lam, 1.0)[0]),
            "arms": out, "best_seconds_to_1e-3": best,
            "plain_fp32_seconds_to_1e-3": plain}


def run_lda(args, rank, world, local_rank):
    """The default line (see the module docstring)."""
    import torch
    from paper_1309_0787_gb300 import otm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    c = dict(LDA)
    k, b, ep = c["k"], c["b"], c["epochs"]
    a0 = k * c["alpha_i"]
    host = lda_inputs(c, rank)
    n = host["X"].shape[0]
    path = LdaPath(otm, torch, c, host, dev)
    otm.sgd_set_form(sgd_form_code(otm, args.sgd_form))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    samples = n * ep
    flops = sym_sgd_flops(n, b, k, ep)
    nsteps = ((n + b - 1) // b) * ep

    for _ in range(args.warmup):
        path.step()
    torch.cuda.synchronize()
    dist_barrier(world)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [{nm: torch.cuda.Event(enable_timing=True) for nm in ("w0", "s0", "s1", "e1")}
          for _ in range(args.steps)]
    l0 = otm.launch_count()
    torch.cuda.synchronize()
    dist_barrier(world)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                       # evict the L2 (129 MB) between steps
        path.step(ev[i])
        ev[i]["e1"].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    dist_barrier(world)
    launches = otm.launch_count() - l0
    clocks = sampler.stop()
    step_ms = [e["w0"].elapsed_time(e["e1"]) for e in ev]
    sgd_ms = [e["s0"].elapsed_time(e["s1"]) for e in ev]
    pre_ms = [e["w0"].elapsed_time(e["s0"]) for e in ev]
    t_max = dist_max(sum(step_ms) / 1e3, world)

    # end to end: inputs in pinned host memory, copies inside the timed region
    X = host["X"]
    pinned = {"X": tuple(torch.from_numpy(a).pin_memory() for a in (X.row_ptr, X.col, X.val)),
              "S": torch.from_numpy(host["S"]).pin_memory(),
              "perm": torch.from_numpy(host["perm"]).pin_memory(),
              "V0t": torch.from_numpy(host["V0"].T.copy()).pin_memory()}
    h2d = sum(a.numel() * a.element_size() for a in pinned["X"])
    h2d += sum(pinned[nm].numel() * pinned[nm].element_size() for nm in ("S", "perm", "V0t"))
    mu_host = torch.empty(c["d"], k, dtype=torch.float64).pin_memory()
    lam_host = torch.empty(k, dtype=torch.float64).pin_memory()
    al_host = torch.empty(k, dtype=torch.float64).pin_memory()
    d2h = (mu_host.numel() + lam_host.numel() + al_host.numel()) * 8
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = max(1, args.steps // 2)
    e2e_ms = 0.0
    path.upload(pinned)       # untimed: the allocator's blocks for the uploaded copies
    path.step()
    torch.cuda.synchronize()
    for i in range(n_e2e):
        flush.fill_(float(i))
        e_start.record()
        path.upload(pinned)
        out = path.step()
        mu_host.copy_(out["comps"], non_blocking=True)
        lam_host.copy_(out["lambda"], non_blocking=True)
        al_host.copy_(out["alpha_hat"], non_blocking=True)
        e_end.record()
        torch.cuda.synchronize()
        e2e_ms += e_start.elapsed_time(e_end)
    e2e_t = dist_max(e2e_ms / 1e3, world)
    path.upload()

    if rank != 0:
        return None
    sgd_avg_s = statistics.mean(sgd_ms) / 1e3
    achieved = flops / sgd_avg_s / 1e12
    line = {
        "metric": METRIC, "value": world * samples * args.steps / t_max, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": c["workload"], "docs": n, "vocabulary": c["d"], "k": k,
                   "nnz": int(X.nnz), "doc_len": "Poisson(300)",
                   "topics": "Dir(0.05) with Zipf skew", "alpha0": a0, "minibatch": b,
                   "epochs": ep, "sgd_steps": nsteps, "samples_per_step": samples,
                   "oversample": c["oversample"], "power_iters": c["power_iters"],
                   "beta0": c["beta0"], "theta": c["theta"],
                   "l2": "flushed between timed steps (256 MiB write); inputs larger than L2",
                   "sgd_form": args.sgd_form,
                   "sgd_split_shape": "%d clusters x %d CTAs" % otm.sgd_split_shape(k, b, True),
                   "parallelism": "replicas" if world > 1 else "single",
                   "host_generation_s": round(host["gen_s"], 1),
                   "corpus_from_cache": host["cached"]},
        "breakdown_ms": {"whiten_project_mean": statistics.mean(pre_ms),
                         "sgd_run": statistics.mean(sgd_ms),
                         "unwhiten": statistics.mean(step_ms) - statistics.mean(pre_ms)
                         - statistics.mean(sgd_ms),
                         "wall_per_step": 1e3 * wall / args.steps},
        "roofline": {"kernel": SGD_KERNEL_NAME.get(args.sgd_form, SGD_KERNEL_NAME["auto"]),
                     "bound": "alu", "achieved": achieved, "peak": FP32_FMA_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_FMA_PEAK_TFLOPS,
                     "traffic": sgd_grid_traffic(args.sgd_form, c),
                     "traffic_source": SGD_GRID_TRAFFIC["capture"] + " (kernel source "
                                       "SHA-256 " + SGD_GRID_TRAFFIC["sha256"][:12] + ")",
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                     "algorithmic_flops_per_launch": flops,
                     "launch_ms": statistics.mean(sgd_ms)},
        "e2e": {"value": world * samples * n_e2e / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(f"bench: timed {args.steps} steps, {1e3 * t_max / args.steps:.2f} ms/step",
          file=sys.stderr, flush=True)
    line["precisions"] = lda_precisions(otm, torch, path, c, host, statistics.mean(sgd_ms))
    print("bench: precision forms done", file=sys.stderr, flush=True)
    line["time_to_1e-3"] = time_to_target(otm, torch, dev)
    print("bench: time to 1e-3 done", file=sys.stderr, flush=True)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = lda_cpu_baseline(c, host)
    return line


def run_stgd(args):
    """The STGD launch alone (one persistent launch = the 20 epochs of the default
    line, 5,860 steps) on the default line's whitened samples, in the FP32 form
    --sgd-form selects: time per launch, samples/s, algorithmic FP32 throughput
    (4 k^2 per sample + 4 k^3 per step) against the derived FP32 peak.  Whitening
    and projection run once, untimed; L2 flushed before each launch."""
    import torch
    from paper_1309_0787_gb300 import otm
    c = dict(LDA)
    dev = torch.device("cuda", 0)
    host = lda_inputs(c, 0)
    path = LdaPath(otm, torch, c, host, dev)
    otm.sgd_set_form(sgd_form_code(otm, args.sgd_form))
    wh, Y, yb3 = path.front()
    n, k, b, ep = Y.shape[0], c["k"], c["b"], c["epochs"]
    a0 = k * c["alpha_i"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one():
        V = path.V0t.clone()
        otm.sgd_run(V, Y, Y, Y, yb3, path.perm, ep, b, c["beta0"], c["theta"], a0)
        return V
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        one()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    otm.sgd_set_form(otm.SGD_FORM_AUTO)
    t = statistics.median(ms) / 1e3
    flops = sym_sgd_flops(n, b, k, ep)
    nsteps = ((n + b - 1) // b) * ep
    return {"metric": "whitened-sample SGD throughput (samples/s), STGD launch alone",
            "value": n * ep / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "stgd_lda_300000_k100_b1024_fp32", "docs": n, "k": k,
                       "minibatch": b, "epochs": ep, "sgd_steps": nsteps,
                       "sgd_form": args.sgd_form,
                       "sgd_split_shape": "%d clusters x %d CTAs" % otm.sgd_split_shape(k, b, True),
                       "l2": "flushed before each launch (256 MiB write)"},
            "us_per_sgd_step": 1e6 * t / nsteps,
            "roofline": {"kernel": SGD_KERNEL_NAME[args.sgd_form], "bound": "alu",
                         "achieved": flops / t / 1e12, "peak": FP32_FMA_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / t / 1e12 / FP32_FMA_PEAK_TFLOPS,
                         "traffic": sgd_grid_traffic(args.sgd_form, c),
                         "traffic_source": SGD_GRID_TRAFFIC["capture"] + " (kernel "
                                           "source SHA-256 " + SGD_GRID_TRAFFIC["sha256"][:12] + ")",
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                         "algorithmic_flops_per_launch": flops},
            "gpu_launches": args.steps, "clocks": clocks}


def run_topic_exact(args):
    """The STGD on the whole third moment of Eq. (3) (self-token terms kept) on the
    default line's corpus, W and M1 from its whitening (untimed), one epoch of
    b = 1,024 documents from the default line's start; L2 flushed before each
    run.  Algorithmic FP32 work per step: 2 k^2 per word occurrence for U = W_g V^T,
    2 k^2 per occurrence and 2 k^2 per document for W_g^T Coef + Y'^T A, plus the
    Gram term 4 k^3 (the sample tensor's 4 k^2 per document for comparison)."""
    import torch
    from paper_1309_0787_gb300 import otm
    c = dict(LDA)
    dev = torch.device("cuda", 0)
    host = lda_inputs(c, 0)
    path = LdaPath(otm, torch, c, host, dev)
    wh, Y, yb3 = path.front()
    n, k, b = Y.shape[0], c["k"], c["b"]
    a0 = k * c["alpha_i"]
    perm = path.perm[:1].contiguous()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one(prec):
        V = path.V0t.clone()
        otm.sgd_run_topic_exact(V, path.Xd, wh["W"], wh["M1"], perm, 1, b, c["beta0"],
                                c["theta"], a0, precision=prec)
        return V

    def timed(prec):
        for _ in range(args.warmup):
            one(prec)
        torch.cuda.synchronize()
        ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            V = one(prec)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms) / 1e3, V
    sampler = ClockSampler(0)
    sampler.start()
    t, V = timed(0)
    t16, V16 = timed(otm.PREC_BF16)
    clocks = sampler.stop()
    # one step on the first minibatch from the start, each form against the FP64 oracle
    from oracle import stgd as ostgd
    docs = host["perm"][0][:b].astype(np.int64)
    Xb = synth.CSR(*_csr_rows(host["X"], docs), (len(docs), host["X"].shape[1]))
    W64 = wh["W"].cpu().numpy().astype(np.float64)
    M164 = wh["M1"].cpu().numpy()
    V0 = host["V0"].astype(np.float64)
    G = ostgd.grad_implicit_topic_exact(V0, Xb, W64, M164, c["theta"], a0)
    gram = ostgd.kappa(c["theta"]) * V0 @ (V0.T @ V0) ** 2
    den = np.linalg.norm(gram) + np.linalg.norm(gram - G)
    step = {}
    for nm, prec in (("fp32", 0), ("bf16", otm.PREC_BF16)):
        V1 = path.V0t.clone()
        otm.sgd_run_topic_exact(V1, otm.DeviceCSR.from_host(Xb, dev), wh["W"], wh["M1"], None, 1,
                                b, c["beta0"], c["theta"], a0, precision=prec)
        Gk = (V0 - V1.cpu().numpy().T.astype(np.float64)) / c["beta0"]
        step[nm] = {"grad_rel_err": float(np.linalg.norm(Gk - G) / den),
                    "grad_rel_err_worst_component": float(
                        (np.linalg.norm(Gk - G, axis=0) /
                         (np.linalg.norm(gram, axis=0) + np.linalg.norm(gram - G, axis=0))).max())}
    nnz = int(host["X"].row_ptr[-1])
    nsteps = (n + b - 1) // b
    flops = 4.0 * k * k * nnz + 2.0 * k * k * n + nsteps * 4.0 * k ** 3
    finite = bool(torch.isfinite(V).all())
    return {"metric": "exact-topic STGD throughput (documents/s), whole Eq. (3)",
            "value": n / t, "unit": "documents/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 accumulation)",
            "data": "synthetic",
            "config": {"workload": "stgd_exact_topic_lda_300000x100000_k100_b1024", "docs": n,
                       "nnz": nnz, "k": k, "minibatch": b, "epochs": 1, "sgd_steps": nsteps,
                       "l2": "flushed before each run (256 MiB write)"},
            "us_per_sgd_step": 1e6 * t / nsteps, "result_finite": finite,
            "bf16": {"ms_per_step": 1e3 * t16, "us_per_sgd_step": 1e6 * t16 / nsteps,
                     "documents_per_s": n / t16, "result_finite": bool(torch.isfinite(V16).all()),
                     "achieved_tflops": flops / t16 / 1e12},
            "one_step_vs_fp64_oracle": step,
            "roofline": {"kernel": "sgd_run_topic_exact (gather, U = W_g V^T, coefficients, "
                                   "W_g^T Coef + Y'^T A, update per step)",
                         "bound": "alu", "achieved": flops / t / 1e12,
                         "peak": FP32_FMA_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops / t / 1e12 / FP32_FMA_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                         "algorithmic_flops_per_run": flops},
            "clocks": clocks}


def _csr_rows(X, rows):
    """(row_ptr, col, val) of the rows `rows` of the CSR X, in that order."""
    lens = (X.row_ptr[rows + 1] - X.row_ptr[rows]).astype(np.int64)
    rp = np.concatenate([[0], np.cumsum(lens)])
    idx = np.concatenate([np.arange(X.row_ptr[r], X.row_ptr[r + 1]) for r in rows])
    return rp, X.col[idx], X.val[idx]


def run_projection(args):
    """The projection y_t = W^T c_t / l_t (Section 3.1) alone, on the default
    line's corpus with a random W (d x k, float32): the gather SpMM's time and
    its achieved bandwidth on the algorithmic HBM bytes 8 nnz (column index and
    count) + 4 (n + 1) (row pointers) + 4 n (row scales) + 4 k n (the output
    rows), against the measured copy bandwidth; the W-row gathers (4 k nnz
    bytes) are served by the L2 and counted apart.  L2 flushed before each call."""
    import torch
    from paper_1309_0787_gb300 import otm
    c = dict(LDA)
    dev = torch.device("cuda", 0)
    host = lda_inputs(c, 0)
    X = host["X"]
    n, d = X.shape
    k = c["k"]
    Xd = otm.DeviceCSR.from_host(X, dev)
    W = torch.from_numpy(synth.gaussian(c["seed"] + 9, d, k)).to(dev)
    invlen = otm.topic_moments(Xd)["row_invlen"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        otm.project(Xd, W, invlen)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        otm.project(Xd, W, invlen)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    t = statistics.median(ms) / 1e3
    nnz = int(X.nnz)
    alg = 8 * nnz + 4 * (n + 1) + 4 * n + 4 * k * n
    gathers = 4 * k * nnz
    return {"metric": "projection throughput (documents/s), gather SpMM", "value": n / t,
            "unit": "documents/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "projection_300000x100000_k100", "docs": n, "vocabulary": d,
                       "k": k, "nnz": nnz, "l2": "flushed before each call (256 MiB write)"},
            "roofline": {"kernel": "spmm_gather_v4_kernel", "bound": "hbm",
                         "achieved": alg / t / 1e9, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                         "frac": alg / t / 1e9 / HBM_PEAK_GBS, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                         "algorithmic_bytes_per_launch": alg},
            "l2_gather_bytes_per_launch": gathers, "l2_gather_gbs": gathers / t / 1e9,
            "gpu_launches": args.steps, "clocks": clocks}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-target", action="store_true",
                    help="batched: skip the time-to-1e-3 comparison")
    ap.add_argument("--workload", default="lda",
                    choices=["lda", "mmsb", "batched", "warmstart", "whitening", "projection",
                             "topic_exact",
                             "stgd"],
                    help="lda: the default line (300,000-document LDA corpus, whole path); "
                         "mmsb: the community-model pipeline; batched: the batched form; "
                         "warmstart: time to 1e-3 with the learned start; whitening: both "
                         "randomised whitening forms on an LDA corpus")
    ap.add_argument("--k", type=int, default=0, help="warmstart: components (default 64)")
    ap.add_argument("--problems", type=int, default=512)
    ap.add_argument("--restarts", type=int, default=8)
    ap.add_argument("--cluster", type=int, default=0,
                    help="batched: CTAs per chain (0 = autotune)")
    ap.add_argument("--sgd-form", default="auto", choices=["auto", "split", "grid", "cluster"],
                    help="lda / mmsb: form of the FP32 STGD kernel")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "batched":
        line = run_batched(args) if rank == 0 else None
    elif args.workload == "warmstart":
        line = run_warmstart(args) if rank == 0 else None
    elif args.workload == "whitening":
        line = run_whitening(args) if rank == 0 else None
    elif args.workload == "projection":
        line = run_projection(args) if rank == 0 else None
    elif args.workload == "topic_exact":
        line = run_topic_exact(args) if rank == 0 else None
    elif args.workload == "stgd":
        line = run_stgd(args) if rank == 0 else None
    elif args.impl == "reference":
        line = (run_lda_reference(args, rank, world) if args.workload == "lda"
                else run_reference(args, rank, world))
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        fn = run_lda if args.workload == "lda" else run_mmsb
        line = fn(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
