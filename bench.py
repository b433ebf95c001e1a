#!/usr/bin/env python
"""Benchmark of the structured-multigrid hot path on GB300.

One step = the whole hot path on one problem: hierarchy set-up (stencil
Galerkin products, smoother set-up, coarsest inverse) followed by the
V-cycle-preconditioned Krylov solve to a relative residual of 1e-9 and the
FP64 true-residual check, with the matrix and right-hand side already in HBM
(the e2e figure adds the host<->device copies).  The metric is time to
solution (lower is better), reported for the FP64 hierarchy (`value`) and
for the FP32 and row-scaled BF16 hierarchies under an FP64 outer iteration
(`forms`, each with its error against the FP64 solution); the V-cycle's
HBM throughput, its per-level cost and the dominant kernel's roofline
fraction are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3]
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
    "c2_128_fp32": dict(desc="aniso27_128^3_ilu0_fw27v_fpcg_fp32hier", dims=(128, 128, 128), gen="q1", smoother=1,
                        transfer=0, precision=1, krylov=1, tol=1e-9),
    # the largest configuration that fits one GPU (56.6 M unknowns), three ways:
    # FP64 hierarchy under PCG (value), FP32 and BF16 hierarchies under FPCG
    "c3": dict(desc="aniso27_384^3_ilu0_fw27v_pcg", dims=(384, 384, 384), gen="q1", smoother=1, transfer=0,
               precision=0, krylov=0, tol=1e-9, forms=(0, 1, 2)),
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
    # the network in place of the finest level's post-smoothing (trained on the
    # residuals the coarse correction leaves; rejected corrections fall back
    # to the skipped post-smoothing)
    "c5_replace": dict(desc="varcoef7_256^3_sgs_fw27v_fpcg_cnn_replaces_post_fp64", dims=(256, 256, 256), gen="fv",
                       smoother=0, transfer=0, precision=0, krylov=1, tol=1e-9,
                       learned=dict(dims=(64, 64, 64), fields=20, pairs=2000, batch=4, lr=1e-3, mode=1)),
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
DEFAULT = "c3"
HBM_PEAK_FALLBACK = 6800.0
FP64_PEAK_NOMINAL = 1.25  # TFLOP/s, used only when the measured figure is missing
FP64_PROBE = os.path.join(ROOT, "profiles", "fp64_fma_peak_gb300.txt")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per point of the
# dominant kernel, from one ncu capture of the current kernel on the same
# problem family at a smaller size (the traffic grows with the points); keyed
# by (kernel, smoother, stencil points, precision).  Absent where no capture
# of the current kernel exists.
TRAFFIC_PER_POINT = {
    # k_sweep3 ILU lower solve, FP64, 27 points: 268.97 MB for 128^3
    ("k_sweep3", 1, 27, 0): (268.970e6 / 128 ** 3, "profiles/k_sweep3_ilu_lower_aniso27_128cubed.md"),
    # k_sweep3h (two warps per strip), same solve: 268.25 MB for 128^3
    ("k_sweep3h", 1, 27, 0): (268.252e6 / 128 ** 3, "profiles/k_sweep3h_ilu_lower_aniso27_128cubed.md"),
}


PREC = {0: "fp64", 1: "fp32", 2: "bf16"}
KRYLOV = {0: "PCG", 1: "FPCG", 2: "FGMRES(30)"}


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
        mgs[-1].set_learned_mode(cfg.get("mode", 0))
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


def fp64_peak():
    """Measured FP64 FMA throughput (TFLOP/s) from the committed probe summary."""
    try:
        for line in open(FP64_PROBE):
            if line.startswith("fp64_tflops:"):
                return float(line.split(":")[1]), "measured FP64 FMA rate of this GPU (independent-FMA probe, CUDA events)"
    except (OSError, ValueError):
        pass
    return FP64_PEAK_NOMINAL, "nominal GB300 FP64 rate (no measurement found)"


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
    st = torch.cuda.current_stream()
    forms = list(w.get("forms", (w["precision"],)))
    main_prec = forms[0]

    def opts(prec):
        # a reduced-precision hierarchy is only approximately symmetric: PCG
        # becomes flexible PCG (FGMRES stays)
        kry = w["krylov"] if (prec == 0 or w["krylov"] == 2) else 1
        return dict(block=B, smoother=w["smoother"], transfer=w["transfer"], precision=prec, krylov=kry, restart=30,
                    sweep_warps=args.sweep_warps)

    theta, learned_info = (None, None)
    if w.get("learned"):
        theta, learned_info = train_post_smoother(w, dev)

    def make_ctx(prec, Amat, lk=logk):
        h = smg.SMG(w["dims"], off, Amat, **opts(prec))
        if theta is not None and prec == main_prec:
            h.set_learned_mode(w["learned"].get("mode", 0))
            h.set_learned_smoother(theta, lk)
        return h

    x = torch.zeros_like(b)

    def step(prec):
        h = make_ctx(prec, A)
        x.zero_()
        it, rr, rc = h.solve(b, x, tol=w["tol"], maxit=1000, check=False)
        s = h.stats()
        h.close()
        if rc != 0:
            raise RuntimeError("solve failed (%s hierarchy): status %d (%s)" % (PREC[prec], rc, smg.strerror(rc)))
        return it, rr, s

    # ---- the main form: W warm-up steps, K timed steps --------------------
    for _ in range(args.warmup):
        step(main_prec)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = smg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with Clocks(dev.index) as clk:
        ev0.record(st)
        for _ in range(args.steps):
            results.append(step(main_prec))
        ev1.record(st)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = smg.launch_count() - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev, world)
    clocks = clk.summary()
    x_main = x.clone()
    form_info = {PREC[main_prec]: {"krylov": KRYLOV[opts(main_prec)["krylov"]],
                                   "time_to_solution_s": round(ms / 1e3, 5), "iterations": results[-1][0],
                                   "final_true_relres": max(r[1] for r in results),
                                   "setup_ms": round(results[-1][2]["setup_ms"], 3), "timed_steps": args.steps}}

    # ---- the other forms: 1 warm-up, a few timed steps, error vs the main form
    for prec in forms[1:]:
        step(prec)
        k = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        res = [step(prec) for _ in range(k)]
        e1.record(st)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(x - x_main) / torch.linalg.vector_norm(x_main))
        form_info[PREC[prec]] = {"krylov": KRYLOV[opts(prec)["krylov"]],
                                 "time_to_solution_s": round(e0.elapsed_time(e1) / k / 1e3, 5),
                                 "iterations": res[-1][0], "final_true_relres": max(r[1] for r in res),
                                 "setup_ms": round(res[-1][2]["setup_ms"], 3), "timed_steps": k,
                                 "rel_error_vs_fp64_solution": err}
    if len(forms) > 1:
        for v in form_info.values():
            v.setdefault("rel_error_vs_fp64_solution", 0.0)
        form_info["error_reference"] = ("the GPU FP64-hierarchy solution of the same problem (its V-cycle and "
                                        "iteration count are parity-checked against the oracle at 128^3 and 256^3)")

    # ---- the same problem with the plain V-cycle and PCG (learned workload) ---
    plain = None
    if theta is not None:
        hp = smg.SMG(w["dims"], off, A, **dict(opts(main_prec), krylov=0))
        hp.close()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        hp = smg.SMG(w["dims"], off, A, **dict(opts(main_prec), krylov=0))
        x.zero_()
        pit, prr, prc = hp.solve(b, x, tol=w["tol"], maxit=1000, check=False)
        hp.close()
        e1.record(st)
        torch.cuda.synchronize()
        if prc != 0:
            raise RuntimeError("plain PCG solve failed: status %d" % prc)
        plain = {"krylov": "PCG", "smoother": "plain V-cycle", "ms": round(e0.elapsed_time(e1), 3),
                 "iterations": pit, "final_true_relres": prr}

    # ---- V-cycle throughput and per-level cost on a persistent hierarchy ----
    z = torch.empty_like(b)
    vcycles = {}
    main_profile = None
    lvl0_warps = 0
    for prec in forms:
        h = smg.SMG(w["dims"], off, A, **opts(prec))
        s = h.stats()
        for _ in range(2):
            h.vcycle(b, z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nv = 5
        e0.record(st)
        for _ in range(nv):
            h.vcycle(b, z)
        e1.record(st)
        torch.cuda.synchronize()
        vc_ms = e0.elapsed_time(e1) / nv
        profs = [h.vcycle_profile(b, z) for _ in range(3)]
        if prec == main_prec and w["smoother"] != 2:
            # which wavefront kernel runs the level-0 sweep the roofline reports
            lvl0_warps = h.level_sweep_warps(0, smg.OP_ILU_LOWER if w["smoother"] == 1 else smg.OP_GS_ZERO)
        h.close()
        stage = {}
        for prof in profs:
            for lvl, name, t in prof:
                stage.setdefault((lvl, name), []).append(t)
        stage = {k: statistics.median(v) for k, v in stage.items()}
        levels = {}
        for (lvl, name), t in sorted(stage.items()):
            e = levels.setdefault(lvl, {"dims": list(s["dims"][lvl]), "sweeps_ms": 0.0, "other_ms": 0.0})
            e["sweeps_ms" if name in ("pre1", "pre2", "post1", "post2") else "other_ms"] += t
        total = sum(e["sweeps_ms"] + e["other_ms"] for e in levels.values())
        per_level = [{"level": lvl, "dims": e["dims"], "sweeps_ms": round(e["sweeps_ms"], 4),
                      "other_ms": round(e["other_ms"], 4),
                      "share": round((e["sweeps_ms"] + e["other_ms"]) / total, 4)} for lvl, e in sorted(levels.items())]
        hbm = float(measured_peaks().get("hbm_gbs", HBM_PEAK_FALLBACK))
        vcycles[PREC[prec]] = {"vcycle_ms": round(vc_ms, 4), "vcycle_bytes": s["vcycle_bytes"],
                               "vcycle_gbs": round(s["vcycle_bytes"] / (vc_ms * 1e-3) / 1e9, 1),
                               "vcycle_hbm_frac": round(s["vcycle_bytes"] / (vc_ms * 1e-3) / 1e9 / hbm, 4),
                               "coarse_levels_share": round(1.0 - per_level[0]["share"], 4), "per_level": per_level}
        if prec == main_prec:
            main_profile = stage
            stats_main = s

    # ---- dominant kernel: the level-0 triangular (or line) sweep of a V-cycle --
    lvl0 = int(w["dims"][0]) * int(w["dims"][1]) * int(w["dims"][2])
    nsf = len(off)
    nlow = nsf // 2
    cbytes = {0: 8, 1: 4, 2: 2}[main_prec]
    vbytes = 8 if main_prec == 0 else 4
    sbytes = 4 if main_prec == 2 else 0
    ny = int(w["dims"][1])
    if w["smoother"] == 2:
        kname = "k_lsweep (line Gauss-Seidel, zero-guess forward, level 0)"
        nz = int(w["dims"][2])
        m = max(2, -(-nz // 128))
        fac_pt = 8.0 * ((m - 1) * 5 + 17) * 128 / nz
        flops_pt, bytes_pt = 2 * (nlow - 1) + 10, nlow * cbytes + fac_pt + 2 * vbytes
    elif w["smoother"] == 1:
        kfile = "k_sweep3h" if lvl0_warps == 2 else "k_sweep3"
        kname = "%s (ILU(0) lower solve, level 0)" % kfile
        flops_pt, bytes_pt = 2 * nlow + 1, nlow * cbytes + 2 * vbytes + sbytes
    else:
        kfile = {2: "k_sweep3h", 1: "k_sweep3"}.get(lvl0_warps, "k_sweep2") if B == 1 else "k_bsweep3"
        kname = "%s (Gauss-Seidel zero-guess forward, level 0)" % kfile
        flops_pt = (2 * nlow + 2) * B * B
        bytes_pt = nlow * cbytes * B * B + vbytes * B * B + 2 * vbytes * B + sbytes
    k_ms = main_profile[(0, "pre1")]
    hbm = float(measured_peaks().get("hbm_gbs", HBM_PEAK_FALLBACK))
    k_gbs = lvl0 * bytes_pt / (k_ms * 1e-3) / 1e9
    tr = TRAFFIC_PER_POINT.get((kfile, w["smoother"], nsf, main_prec)) if B == 1 and w["smoother"] != 2 else None
    traffic = None if tr is None else round(tr[0] * lvl0)
    hbm_roof = {"achieved": round(k_gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(k_gbs / hbm, 4),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in measured_peaks()
                else "fallback", "algorithmic_bytes_per_point": bytes_pt}
    common = {"traffic": traffic, "kernel": kname, "launch_ms": round(k_ms, 4),
              "launch_timing": "CUDA events around the kernel inside a profiled V-cycle (median of 3)"}
    if tr is not None:
        common["traffic_source"] = "ncu capture of the same kernel at a smaller size (%s), scaled by the points" % tr[1]
    if main_prec == 0:
        # FP64: the binding roof is the FP64 pipe whenever its time at the
        # measured rate exceeds the bytes' time at the measured bandwidth
        pk, src = fp64_peak()
        k_tf = lvl0 * flops_pt / (k_ms * 1e-3) / 1e12
        alu_roof = {"achieved": round(k_tf, 4), "peak": pk, "unit": "TFLOP/s", "frac": round(k_tf / pk, 4),
                    "peak_source": src, "algorithmic_flops_per_point": flops_pt}
        if flops_pt / (pk * 1e12) > bytes_pt / (hbm * 1e9):
            roof = dict({"bound": "alu"}, **alu_roof, **common, hbm=hbm_roof)
        else:
            roof = dict({"bound": "hbm"}, **hbm_roof, **common, alu=alu_roof)
    else:
        roof = dict({"bound": "hbm"}, **hbm_roof, **common)

    extra = {"forms": form_info, "vcycle": vcycles}
    if learned_info is not None:
        extra.update({"learned": learned_info, "plain_pcg": plain})
    out = dict(ms=ms, iters=results[-1][0], relres=max(r[1] for r in results), stats=stats_main, clocks=clocks,
               launches=launches, roof=roof, hbm=hbm, extra=extra, e2e_ms=float("nan"), h2d=0, d2h=0)
    if args.no_e2e:
        return out

    # ---- e2e: host buffers, copies inside the timed region (main form) ------
    A_h = A.cpu().pin_memory()
    b_h = b.cpu().pin_memory()
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    A_d = torch.empty_like(A)
    b_d = torch.empty_like(b)
    x_d = torch.empty_like(b)
    lk_h = None if logk is None else logk.cpu().pin_memory()
    lk_d = None if logk is None else torch.empty_like(logk)

    phase = []  # per step: (start, copies in, solved, copied out) events

    def e2e_step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(st)
        A_d.copy_(A_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        if lk_d is not None:
            lk_d.copy_(lk_h, non_blocking=True)
        ev[1].record(st)
        hh = make_ctx(main_prec, A_d, lk_d)
        x_d.zero_()
        it, rr, rc = hh.solve(b_d, x_d, tol=w["tol"], maxit=1000, check=False)
        hh.close()
        if rc != 0:
            raise RuntimeError("e2e solve failed: status %d" % rc)
        ev[2].record(st)
        x_h.copy_(x_d, non_blocking=True)
        ev[3].record(st)
        phase.append(ev)

    e2e_step()
    torch.cuda.synchronize()
    ne = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(ne):
        e2e_step()
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ne
    e2e_wall = (time.perf_counter() - t0) / ne * 1e3
    h2d = A.numel() * 8 + n * 8 + (0 if logk is None else logk.numel() * 8)
    timed = phase[-ne:]
    cin = sum(ev[0].elapsed_time(ev[1]) for ev in timed) / ne
    comp = sum(ev[1].elapsed_time(ev[2]) for ev in timed) / ne
    cout = sum(ev[2].elapsed_time(ev[3]) for ev in timed) / ne
    out.update(e2e_ms=max_over_ranks(max(e2e_ms, e2e_wall), dev, world), h2d=h2d, d2h=n * 8,
               e2e_phases={"h2d_ms": round(cin, 3), "h2d_gbs": round(h2d / (cin * 1e-3) / 1e9, 1),
                           "setup_and_solve_ms": round(comp, 3), "d2h_ms": round(cout, 3),
                           "wall_ms": round(e2e_wall, 3), "events_ms": round(e2e_ms, 3)})
    return out


def oracle_sample(w, seed=0, full_iters=None):
    """Times the CPU oracle (one thread) on a bounded sample of the workload:
    the same problem family on a grid with 1/8 of the points per dimension
    halving (at most 64^3 points), full set-up plus Krylov solve.  The set-up
    is scaled to the workload by the number of unknowns, the solve by the
    unknowns and, when the full-size iteration count is known, by the ratio of
    iteration counts."""
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
    prec = w["precision"] if (B == 1 or w["precision"] != 2) else 0
    t0 = time.perf_counter()
    mg = orc.MG(sd, off, A.reshape(A.shape[0], -1) if B == 1 else A, B=B, smoother=w["smoother"],
                transfer=w["transfer"], precision=prec)
    t1 = time.perf_counter()
    if w["krylov"] == 2:
        x, rc, it, rr, _ = mg.fgmres(b, tol=w["tol"], restart=30, maxit=1000)
    else:
        x, rc, it, rr, _ = mg.pcg(b, tol=w["tol"], maxit=1000, flexible=w["krylov"] == 1)
    t2 = time.perf_counter()
    scale = full / (sd[0] * sd[1] * sd[2])
    ratio = (full_iters / it) if (full_iters and it) else 1.0
    return dict(value=(t1 - t0) * scale + (t2 - t1) * scale * ratio, raw_s=t2 - t0, setup_s=t1 - t0, solve_s=t2 - t1,
                scale=scale, iter_ratio=ratio, grid=sd, iters=it, relres=rr, rc=rc)


def sample_text(o, full_iters=None):
    txt = ("grid %s (1/%d of the unknowns): set-up %.2f s + solve %.2f s in %d iterations on one core; set-up x%d, "
           "solve x%d" % ("x".join(map(str, o["grid"])), o["scale"], o["setup_s"], o["solve_s"], o["iters"], o["scale"],
                          o["scale"]))
    if full_iters:
        txt += " x %d/%d (iterations at full size / in the sample)" % (full_iters, o["iters"])
    else:
        txt += " (iteration growth with size not included: a lower bound)"
    return txt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    ap.add_argument("--sweep-warps", type=int, default=0, choices=[0, 1, 2],
                    help="warps per strip of the wavefront sweeps (0: the library's choice)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    metric = "time to solution (set-up + Krylov to rel-res %g), %s" % (w["tol"], w["desc"])
    config = {"workload": w["desc"], "dims": list(w["dims"]), "unknowns_per_point": w.get("block", 1),
              "smoother": ["sym-GS", "ILU(0)", "sym-LGS (z-lines)"][w["smoother"]], "transfer": ["3d27v", "3d8c", "3d64c interp. + 3d8c restr.",
                                                                "x-y semi-coarsening, 2d16c interp. + 2d4c restr."][w["transfer"]],
              "hierarchy_precision": "+".join(["fp64", "fp32", "bf16-rowscaled"][p] for p in w.get("forms", (w["precision"],))),
              "krylov": ["PCG", "FPCG", "FGMRES(30)"][w["krylov"]], "tol": w["tol"],
              "parallelism": "replicas" if args.gpus > 1 else "single-gpu",
              "l2": "inputs larger than L2 (matrix of %.1f GB)" % (
                  w["dims"][0] * w["dims"][1] * w["dims"][2] * 8 * (27 if w["gen"] in ("q1", "q1z") else 7) *
                  w.get("block", 1) ** 2 / 1e9)}
    if args.impl == "reference":
        if rank != 0:
            return
        # each step is one bounded oracle sample of the workload
        for _ in range(args.warmup):
            oracle_sample(w)
        runs = [oracle_sample(w) for _ in range(max(1, args.steps))]
        raw = statistics.mean(o["raw_s"] for o in runs)
        value = statistics.median(o["value"] for o in runs)
        o = runs[-1]
        line = {"impl": "reference", "metric": metric, "value": round(value, 4), "unit": "s", "n_gpus": args.gpus,
                "steps": len(runs), "warmup": args.warmup, "ms_per_step": round(raw * 1e3, 2),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "sample_grid": list(o["grid"]), "sample_s": round(raw, 4), "scale_unknowns": o["scale"],
                "value_is": "median over the steps of the sample time scaled to the workload's unknowns; "
                            "ms_per_step is the unscaled sample time",
                "cpu_baseline": {"value": round(value, 4), "unit": "s", "cores": 1, "kind": "oracle",
                                 "sample": sample_text(o)},
                "e2e": {"value": round(value, 4), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
        o = oracle_sample(w, full_iters=r["iters"])
        cpu = {"value": round(o["value"], 3), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": sample_text(o, r["iters"])}
        if w.get("learned"):
            cpu["sample"] += "; plain V-cycle (the timed oracle runs no network)"
    s = r["stats"]
    main = PREC[w.get("forms", (w["precision"],))[0]]
    vc = r["extra"]["vcycle"][main]
    line = {"metric": metric, "value": round(r["ms"] / 1e3, 5), "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(r["ms"], 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+bf16"}[main],
            "data": "synthetic", "config": config,
            "iterations": r["iters"], "final_true_relres": r["relres"],
            "setup_ms": round(s["setup_ms"], 3), "levels": s["levels"],
            "grid_complexity": round(s["grid_complexity"], 4), "operator_complexity": round(s["operator_complexity"], 4),
            "vcycle_ms": vc["vcycle_ms"], "vcycle_gbs": vc["vcycle_gbs"], "vcycle_hbm_frac": vc["vcycle_hbm_frac"],
            "roofline": r["roof"],
            "cpu_baseline": cpu,
            "e2e": dict({"value": round(r["e2e_ms"] / 1e3, 5), "unit": "s", "h2d_bytes_per_step": int(r["h2d"]),
                         "d2h_bytes_per_step": int(r["d2h"])}, **({"phases": r["e2e_phases"]} if "e2e_phases" in r else {})),
            "gpu_launches": int(r["launches"]), "clocks": r["clocks"]}
    line.update(r.get("extra", {}))
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
