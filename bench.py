#!/usr/bin/env python
"""Benchmark of the structured-multigrid hot path on GB300.

One step = the whole hot path on one problem: hierarchy set-up (stencil
Galerkin products, smoother set-up, coarsest inverse) followed by the
V-cycle-preconditioned Krylov solve to a relative residual of 1e-9 and the
FP64 true-residual check, with the matrix and right-hand side already in HBM
(the e2e figure adds the host<->device copies).  The metric is time to
solution (lower is better); the V-cycle's HBM throughput and the dominant
kernel's roofline fraction are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2]
  python bench.py --impl reference     (CPU oracle on a bounded sample)
Multi-GPU runs are independent replicas (one problem per GPU, no collective
on the data path); the reported time is the maximum over ranks.
"""
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

WORKLOADS = {
    # 3D 7-point Poisson, 32^3, symmetric GS V(1,1), PCG (L2-resident)
    "c1": dict(desc="poisson7_32^3_sgs_fw27v_pcg_fp64", dims=(32, 32, 32), gen="lap", smoother=0, transfer=0,
               precision=0, krylov=0, tol=1e-9),
    # 27-point anisotropic Q1 diffusion, 256^3, ILU(0), PCG, FP64 (the headline workload)
    "c2": dict(desc="aniso27_256^3_ilu0_fw27v_pcg_fp64", dims=(256, 256, 256), gen="q1", smoother=1, transfer=0,
               precision=0, krylov=0, tol=1e-9),
    # the same problem at 128^3: the small case for detailed profiles (matrix 453 MB > L2)
    "c2_128": dict(desc="aniso27_128^3_ilu0_fw27v_pcg_fp64", dims=(128, 128, 128), gen="q1", smoother=1,
                   transfer=0, precision=0, krylov=0, tol=1e-9),
    "c3_fp64": dict(desc="aniso27_384^3_ilu0_pcg_fp64", dims=(384, 384, 384), gen="q1", smoother=1, transfer=0,
                    precision=0, krylov=0, tol=1e-9),
    "c3_fp32": dict(desc="aniso27_384^3_ilu0_fpcg_fp32hier", dims=(384, 384, 384), gen="q1", smoother=1,
                    transfer=0, precision=1, krylov=1, tol=1e-9),
    "c3_bf16": dict(desc="aniso27_384^3_ilu0_fpcg_bf16hier", dims=(384, 384, 384), gen="q1", smoother=1,
                    transfer=0, precision=2, krylov=1, tol=1e-9),
    "c2_fp32": dict(desc="aniso27_256^3_ilu0_fpcg_fp32hier", dims=(256, 256, 256), gen="q1", smoother=1,
                    transfer=0, precision=1, krylov=1, tol=1e-9),
    "c2_bf16": dict(desc="aniso27_256^3_ilu0_fpcg_bf16hier", dims=(256, 256, 256), gen="q1", smoother=1,
                    transfer=0, precision=2, krylov=1, tol=1e-9),
    "c4": dict(desc="block3x3_7pt_128x128x64_bsgs_pc8c_fgmres30_fp64", dims=(128, 128, 64), gen="blk", smoother=0,
               transfer=1, precision=0, krylov=2, tol=1e-8, block=3),
    "c4_fp32": dict(desc="block3x3_7pt_128x128x64_bsgs_pc8c_fgmres30_fp32hier", dims=(128, 128, 64), gen="blk",
                    smoother=0, transfer=1, precision=1, krylov=2, tol=1e-8, block=3),
    # learned post-smoother: trained on 64^3 fields (2000 pairs), evaluated on
    # an unseen field at 256^3 with FPCG; the plain GS V-cycle PCG solve of the
    # same problem is timed beside it
    "c5": dict(desc="varcoef7_256^3_sgs_fw27v_fpcg_cnn_fp64", dims=(256, 256, 256), gen="fv", smoother=0,
               transfer=0, precision=0, krylov=1, tol=1e-9, learned=dict(dims=(64, 64, 64), fields=20, pairs=2000,
                                                                          batch=4, lr=1e-3)),
    "c5_plain": dict(desc="varcoef7_256^3_sgs_fw27v_pcg_fp64", dims=(256, 256, 256), gen="fv", smoother=0,
                     transfer=0, precision=0, krylov=0, tol=1e-9),
    # the same cell-centred variable-coefficient 7-point matrix with ILU(0) and
    # the cell-centred transfer pair (3d64c interpolation, 3d8c restriction:
    # Table 8's rhd-3T setting), whose V-cycle is nonsymmetric -> FPCG / FGMRES;
    # c6_fw27v is the vertex pair on the same problem for comparison
    "c6": dict(desc="varcoef7_256^3_ilu0_c64c_fpcg_fp64", dims=(256, 256, 256), gen="fv", smoother=1, transfer=2,
               precision=0, krylov=1, tol=1e-9),
    "c6_fgmres": dict(desc="varcoef7_256^3_ilu0_c64c_fgmres30_fp64", dims=(256, 256, 256), gen="fv", smoother=1,
                      transfer=2, precision=0, krylov=2, tol=1e-9),
    "c6_fw27v": dict(desc="varcoef7_256^3_ilu0_fw27v_fpcg_fp64", dims=(256, 256, 256), gen="fv", smoother=1,
                     transfer=0, precision=0, krylov=1, tol=1e-9),
    # 27-point Q1 diffusion with the strong coupling along z (k = 1e-3, 1e-3,
    # 1): symmetric line Gauss-Seidel along z (Sec. 4.4 LGS), PCG
    "c7": dict(desc="zaniso27_256^3_lgs_fw27v_pcg_fp64", dims=(256, 256, 256), gen="q1z", smoother=2, transfer=0,
               precision=0, krylov=0, tol=1e-9),
    "c7_128": dict(desc="zaniso27_128^3_lgs_fw27v_pcg_fp64", dims=(128, 128, 128), gen="q1z", smoother=2,
                   transfer=0, precision=0, krylov=0, tol=1e-9),
    # the same matrix with 2-D semi-coarsening in x and y (2d4c / 2d16c) and
    # z-line smoothing under FGMRES(30): Table 8's weather setting
    "c8": dict(desc="zaniso27_256^3_lgs_semicoarse_xy_fgmres30_fp64", dims=(256, 256, 256), gen="q1z", smoother=2,
               transfer=3, precision=0, krylov=2, tol=1e-9),
}
DEFAULT = "c2"
HBM_PEAK_FALLBACK = 6800.0
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (no FP64 tensor path)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_problem(w, seed, device, with_logk=False):
    from paper_2506_21932_gb300 import inputs as I
    d = w["dims"]
    n = d[0] * d[1] * d[2]
    B = w.get("block", 1)
    logk = None
    if w["gen"] == "lap":
        off, A = I.OFF7, I.laplace7(d, device=device)
    elif w["gen"] == "q1":
        off, A = I.OFF27, I.q1_aniso27(d, seed, device=device)
    elif w["gen"] == "q1z":
        off, A = I.OFF27, I.q1_aniso27(d, seed, aniso=(1e-3, 1e-3, 1.0), device=device)
    elif w["gen"] == "fv":
        off, (A, logk) = I.OFF7, I.varcoef7(d, seed, device=device)
    else:
        off, A = I.OFF7, I.block7_layered(d, seed, device=device)
    b = I.rhs(n * B, 1000 + seed, device=device)
    if with_logk:
        return off, A.contiguous(), b.contiguous(), (None if logk is None else logk.contiguous())
    return off, A.contiguous(), b.contiguous()


def train_post_smoother(w, dev):
    """Trains the learned post-smoother on seeded 64^3 fields (training seeds
    1000 + f) with the library's own kernels; returns (theta, info)."""
    import torch
    from paper_2506_21932_gb300 import smg
    from paper_2506_21932_gb300.learned import PostSmootherTrainer
    cfg = w["learned"]
    tw = dict(w, dims=cfg["dims"])
    mgs, lks = [], []
    for f in range(cfg["fields"]):
        off, A, _, logk = make_problem(tw, 1000 + f, dev, with_logk=True)
        mgs.append(smg.SMG(cfg["dims"], off, A, smoother=w["smoother"], transfer=w["transfer"], krylov=1))
        lks.append(logk)
    tr = PostSmootherTrainer(mgs, lks, seed=0, lr=cfg["lr"], batch=cfg["batch"])
    loss0 = tr.eval_loss(8)
    steps = cfg["pairs"] // cfg["batch"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = tr.train(steps)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    loss1 = tr.eval_loss(8)
    theta = tr.theta.clone()
    for m in mgs:
        m.close()
    return theta, {"train_s": round(train_s, 3), "pairs": steps * cfg["batch"], "fields": cfg["fields"],
                   "grid": list(cfg["dims"]), "loss_before": round(loss0, 6), "loss_after": round(loss1, 6),
                   "loss_last_steps": round(sum(losses[-20:]) / min(20, len(losses)), 6)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[t] for r in rows for t in range(4) if r[5 + t].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x, device, world):
    """Replicas: the job takes as long as its slowest rank (one process per
    GPU, each solving its own problem); a no-op on one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, w, rank, world):
    import torch
    from paper_2506_21932_gb300 import smg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    smg.lib()
    B = w.get("block", 1)
    off, A, b, logk = make_problem(w, rank, dev, with_logk=True)
    n = b.numel()
    x = torch.zeros_like(b)
    st = torch.cuda.current_stream()
    kw = dict(block=B, smoother=w["smoother"], transfer=w["transfer"], precision=w["precision"],
              krylov=w["krylov"], restart=30)
    theta, learned_info = (None, None)
    if w.get("learned"):
        theta, learned_info = train_post_smoother(w, dev)

    def make_ctx(Amat, lk=logk):
        h = smg.SMG(w["dims"], off, Amat, **kw)
        if theta is not None:
            h.set_learned_smoother(theta, lk)
        return h

    def step():
        h = make_ctx(A)
        x.zero_()
        it, rr, rc = h.solve(b, x, tol=w["tol"], maxit=1000, check=False)
        s = h.stats()
        h.close()
        return it, rr, rc, s

    for _ in range(args.warmup):
        it, rr, rc, s = step()
    if rc != 0:
        raise RuntimeError("solve failed: status %d (%s)" % (rc, smg.strerror(rc)))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = smg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with Clocks(dev.index) as clk:
        ev0.record(st)
        for _ in range(args.steps):
            results.append(step())
        ev1.record(st)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = smg.launch_count() - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev, world)
    iters = [r[0] for r in results]
    relres = max(r[1] for r in results)
    s = results[-1][3]
    clocks = clk.summary()

    # --- the same problem with the plain V-cycle and PCG, for comparison ------
    plain = None
    if theta is not None:
        hp = smg.SMG(w["dims"], off, A, **dict(kw, krylov=0))
        hp.close()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        hp = smg.SMG(w["dims"], off, A, **dict(kw, krylov=0))
        x.zero_()
        pit, prr, prc = hp.solve(b, x, tol=w["tol"], maxit=1000, check=False)
        hp.close()
        e1.record(st)
        torch.cuda.synchronize()
        plain = {"krylov": "PCG", "smoother": "plain GS V-cycle", "ms": round(e0.elapsed_time(e1), 3),
                 "iterations": pit, "final_true_relres": prr, "status": prc}

    # --- V-cycle throughput on a persistent hierarchy (plain V-cycle) ----------
    h = smg.SMG(w["dims"], off, A, **kw)
    z = torch.empty_like(b)
    for _ in range(2):
        h.vcycle(b, z)
    torch.cuda.synchronize()
    nv = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(nv):
        h.vcycle(b, z)
    e1.record(st)
    torch.cuda.synchronize()
    vc_ms = e0.elapsed_time(e1) / nv
    vc_gbs = s["vcycle_bytes"] / (vc_ms * 1e-3) / 1e9

    # --- dominant kernel: level-0 lower triangular sweep, timed live -----------
    lvl0 = int(w["dims"][0]) * int(w["dims"][1]) * int(w["dims"][2])
    nsf = len(off)
    nlow = nsf // 2
    cbytes = {0: 8, 1: 4, 2: 2}[w["precision"]]
    vbytes = 8 if w["precision"] == 0 else 4
    if w["precision"] == 0:
        vec = torch.empty(lvl0 * B, dtype=torch.float64, device=dev)
        rhs = b
    else:
        vec = torch.empty(lvl0 * B, dtype=torch.float32, device=dev)
        rhs = b.float()
    ny = int(w["dims"][1])
    kfile = ("k_sweep3" if ny <= 512 else "k_sweep2") if B == 1 else ("k_bsweep3" if ny <= 512 else "k_sweep (3x3 blocks)")
    if w["smoother"] == 2:
        op, kname = smg.OP_LGS_FORWARD, "k_lsweep (line Gauss-Seidel forward, level 0)"
        # column factors: 128 chunks of m rows, 5 doubles per chunk row after the
        # first and 17 per chunk, per column of nz points
        nz = int(w["dims"][2])
        m = max(2, -(-nz // 128))
        fac_pt = 8.0 * ((m - 1) * 5 + 17) * 128 / nz
        flops_pt, bytes_pt = 2 * (nsf - 3) + 10, nsf * cbytes + fac_pt + 3 * vbytes
        vec.zero_()
        run_k = lambda: h.level_apply(0, op, x=vec, b=rhs)
    elif w["smoother"] == 1:
        op, kname = smg.OP_ILU_LOWER, "%s (ILU(0) lower solve, level 0)" % kfile
        flops_pt, bytes_pt = 2 * nlow + 1, nlow * cbytes + 2 * vbytes + (4 if w["precision"] == 2 else 0)
        run_k = lambda: h.level_apply(0, op, b=rhs, y=vec)
    else:
        op, kname = smg.OP_GS_FORWARD, "%s (Gauss-Seidel forward, level 0)" % kfile
        flops_pt = (2 * (nsf - 1) + 2) * B * B
        bytes_pt = ((nsf - 1) * cbytes * B * B + (8 if w["precision"] == 0 else 4) * B * B + 3 * vbytes * B
                    + (4 if w["precision"] == 2 else 0))
        vec.zero_()
        run_k = lambda: h.level_apply(0, op, x=vec, b=rhs)
    for _ in range(2):
        run_k()
    nk = 10
    e0.record(st)
    for _ in range(nk):
        run_k()
    e1.record(st)
    torch.cuda.synchronize()
    k_ms = e0.elapsed_time(e1) / nk
    h.close()
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    k_gbs = lvl0 * bytes_pt / (k_ms * 1e-3) / 1e9
    k_tf = lvl0 * flops_pt / (k_ms * 1e-3) / 1e12
    fp64 = w["precision"] == 0
    # DRAM bytes per launch of the dominant kernel from one ncu capture
    # (dram__bytes_read.sum + dram__bytes_write.sum) of the same kernel on the
    # same problem at 128^3, scaled by the 8x points of a 256^3 launch; None
    # where no capture of the current kernel exists
    traffic = {"c2": round(8 * (483.681536e6 + 16.680960e6))}.get(args.workload)
    if fp64:
        roof = {"bound": "alu", "achieved": round(k_tf, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(k_tf / FP64_PEAK_TFLOPS, 4), "traffic": traffic, "kernel": kname,
                "peak_source": "nominal GB300 FP64 rate 1.25 TFLOP/s (no FP64 tensor path)",
                "hbm_achieved_gbs": round(k_gbs, 1), "hbm_frac_of_measured": round(k_gbs / hbm, 4),
                "algorithmic_flops_per_point": flops_pt, "algorithmic_bytes_per_point": bytes_pt,
                "launch_ms": round(k_ms, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(k_gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(k_gbs / hbm, 4), "traffic": traffic, "kernel": kname,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_point": bytes_pt, "launch_ms": round(k_ms, 4)}

    extra = {}
    if learned_info is not None:
        extra = {"learned": learned_info, "plain_pcg": plain}
    if args.no_e2e:
        return dict(ms=ms, iters=iters, relres=relres, stats=s, clocks=clocks, launches=launches, vc_ms=vc_ms,
                    vc_gbs=vc_gbs, hbm=hbm, roof=roof, e2e_ms=float("nan"), h2d=0, d2h=0, extra=extra)

    # --- e2e: host buffers, copies inside the timed region ---------------------
    A_h = A.cpu().pin_memory()
    b_h = b.cpu().pin_memory()
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    A_d = torch.empty_like(A)
    b_d = torch.empty_like(b)
    x_d = torch.empty_like(b)
    lk_h = None if logk is None else logk.cpu().pin_memory()
    lk_d = None if logk is None else torch.empty_like(logk)

    def e2e_step():
        A_d.copy_(A_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        if lk_d is not None:
            lk_d.copy_(lk_h, non_blocking=True)
        hh = make_ctx(A_d, lk_d)
        x_d.zero_()
        hh.solve(b_d, x_d, tol=w["tol"], maxit=1000, check=False)
        hh.close()
        x_h.copy_(x_d, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ne = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    e0.record(st)
    for _ in range(ne):
        e2e_step()
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ne
    e2e_wall = (time.perf_counter() - t0) / ne * 1e3
    e2e_ms = max_over_ranks(max(e2e_ms, e2e_wall), dev, world)

    return dict(ms=ms, iters=iters, relres=relres, stats=s, clocks=clocks, launches=launches, vc_ms=vc_ms,
                vc_gbs=vc_gbs, hbm=hbm, roof=roof, e2e_ms=e2e_ms,
                h2d=A.numel() * 8 + n * 8 + (0 if logk is None else logk.numel() * 8), d2h=n * 8, extra=extra)


def oracle_sample(w, seed=0):
    """Times the CPU oracle on a bounded sample of the workload: the same
    problem family on a grid with 1/8 (or 1/64) of the points, full set-up plus
    Krylov solve, scaled to the workload by the number of unknowns."""
    import numpy as np
    from oracle import oracle as orc
    orc.build()
    orc.set_threads(1)  # the oracle as written: one thread
    d = w["dims"]
    full = d[0] * d[1] * d[2]
    shrink = 1
    while full // shrink ** 3 > 64 ** 3 and min(d) // (2 * shrink) >= 8:
        shrink *= 2
    sd = tuple(max(4, t // shrink) for t in d)
    ws = dict(w, dims=sd)
    off, A, b = make_problem(ws, seed, "cpu")
    A, b = A.numpy(), b.numpy()
    B = w.get("block", 1)
    t0 = time.perf_counter()
    # the oracle's reduced-precision cycles are scalar only: a block workload
    # is timed with its FP64 hierarchy
    prec = w["precision"] if B == 1 else 0
    mg = orc.MG(sd, off, A.reshape(A.shape[0], -1) if B == 1 else A, B=B, smoother=w["smoother"],
                transfer=w["transfer"], precision=prec)
    if w["krylov"] == 2:
        x, rc, it, rr, _ = mg.fgmres(b, tol=w["tol"], restart=30, maxit=1000)
    else:
        x, rc, it, rr, _ = mg.pcg(b, tol=w["tol"], maxit=1000, flexible=w["krylov"] == 1)
    t = time.perf_counter() - t0
    scale = full / (sd[0] * sd[1] * sd[2])
    return dict(value=t * scale, raw_s=t, scale=scale, grid=sd, iters=it, relres=rr, rc=rc,
                fp64_hierarchy=prec != w["precision"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    metric = "time to solution (set-up + Krylov to rel-res %g), %s" % (w["tol"], w["desc"])
    config = {"workload": w["desc"], "dims": list(w["dims"]), "unknowns_per_point": w.get("block", 1),
              "smoother": ["sym-GS", "ILU(0)", "sym-LGS (z-lines)"][w["smoother"]], "transfer": ["3d27v", "3d8c", "3d64c interp. + 3d8c restr.",
                                                                "x-y semi-coarsening, 2d16c interp. + 2d4c restr."][w["transfer"]],
              "hierarchy_precision": ["fp64", "fp32", "bf16-rowscaled"][w["precision"]],
              "krylov": ["PCG", "FPCG", "FGMRES(30)"][w["krylov"]], "tol": w["tol"],
              "parallelism": "replicas" if args.gpus > 1 else "single-gpu",
              "l2": "inputs larger than L2 (matrix of %.1f GB)" % (
                  w["dims"][0] * w["dims"][1] * w["dims"][2] * 8 * (27 if w["gen"] in ("q1", "q1z") else 7) *
                  w.get("block", 1) ** 2 / 1e9)}
    if args.impl == "reference":
        if rank != 0:
            return
        r = oracle_sample(w)
        line = {"impl": "reference", "metric": metric, "value": round(r["value"], 4), "unit": "s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["value"] * 1e3, 2),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": round(r["value"], 4), "unit": "s", "cores": 1, "kind": "oracle",
                                 "sample": "grid %s (1/%d of the unknowns), full set-up + solve (%d iterations), "
                                           "time x%d" % ("x".join(map(str, r["grid"])), r["scale"], r["iters"],
                                                         r["scale"])},
                "e2e": {"value": round(r["value"], 4), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    r = run_ours(args, w, rank, world)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        o = oracle_sample(w)
        cpu = {"value": round(o["value"], 3), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": "grid %s (1/%d of the unknowns), full set-up + solve in %d iterations, time x%d" % (
                   "x".join(map(str, o["grid"])), o["scale"], o["iters"], o["scale"])}
        if w.get("learned"):
            cpu["sample"] += "; plain V-cycle (the timed oracle runs no network)"
        if o.get("fp64_hierarchy"):
            cpu["sample"] += "; FP64 hierarchy (the oracle has no reduced-precision block cycle)"
    s = r["stats"]
    line = {"metric": metric, "value": round(r["ms"] / 1e3, 5), "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(r["ms"], 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f64+f32", "f64+bf16"][w["precision"]], "data": "synthetic",
            "config": config,
            "iterations": r["iters"][-1], "final_true_relres": r["relres"],
            "setup_ms": round(s["setup_ms"], 3), "levels": s["levels"],
            "grid_complexity": round(s["grid_complexity"], 4), "operator_complexity": round(s["operator_complexity"], 4),
            "vcycle_ms": round(r["vc_ms"], 4), "vcycle_gbs": round(r["vc_gbs"], 1),
            "vcycle_hbm_frac": round(r["vc_gbs"] / r["hbm"], 4),
            "roofline": r["roof"],
            "cpu_baseline": cpu,
            "e2e": {"value": round(r["e2e_ms"] / 1e3, 5), "unit": "s", "h2d_bytes_per_step": int(r["h2d"]),
                    "d2h_bytes_per_step": int(r["d2h"])},
            "gpu_launches": int(r["launches"]), "clocks": r["clocks"]}
    line.update(r.get("extra", {}))
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
