"""The benchmark's reference arm (the CPU oracle on a bounded sample of a
workload) runs without a GPU and prints one JSON line with the contract's
keys; the GPU arm's configuration labels cover every workload."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("poisson7_32^3")
    # the steps it reports are the samples it ran; the per-step time is the
    # unscaled sample time, reported beside the scale
    assert d["steps"] == 1 and abs(d["ms_per_step"] - 1e3 * d["sample_s"]) <= 1e-3 * max(1.0, d["ms_per_step"])
    assert d["scale_unknowns"] >= 1 and d["value"] >= 0.99 * d["sample_s"] * d["scale_unknowns"] / 10


def test_every_workload_has_a_label():
    sys.path.insert(0, ROOT)
    import bench
    for name, w in bench.WORKLOADS.items():
        assert w["smoother"] in (0, 1, 2) and w["transfer"] in (0, 1, 2, 3) and w["krylov"] in (0, 1, 2), name
        assert w["gen"] in ("lap", "q1", "q1z", "fv", "blk"), name
        assert len(w["dims"]) == 3 and w["tol"] > 0, name


def test_traffic_constants_trace_to_the_committed_profiles():
    """Every DRAM-bytes-per-point constant bench.py reports as
    roofline.traffic is the dram read + write of the ncu summary it cites,
    divided by the points of that capture (128^3), and stays within 1.2x of
    the kernel's algorithmic bytes (a larger figure would mean re-reads)."""
    import importlib.util
    import re
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.TRAFFIC_PER_POINT
    for (kernel, smoother, ns, prec), (per_point, src) in bench.TRAFFIC_PER_POINT.items():
        path = os.path.join(ROOT, src)
        assert os.path.exists(path), src
        text = open(path).read()
        assert kernel in text.splitlines()[0], (kernel, src)
        m = re.search(r"\| dram read / write \| ([0-9.]+) MB / ([0-9.]+) MB", text)
        assert m, src
        captured = (float(m.group(1)) + float(m.group(2))) * 1e6 / 128 ** 3
        assert abs(captured - per_point) <= 2e-3 * per_point, (src, captured, per_point)
        # ILU(0) lower solve: n_low coefficients + b + u per point
        assert smoother == 1 and ns == 27
        c = {0: 8, 1: 4, 2: 2}[prec]
        algorithmic = 13 * c + 2 * (8 if prec == 0 else 4) + (4 if prec == 2 else 0)
        assert algorithmic <= per_point <= 1.2 * algorithmic, (src, per_point, algorithmic)
