"""Benchmark: crack-length-controlled increments of a 512 x 512 fibre composite on GB300.

A step is one crack-length increment (Algorithm 2): Newton iterations, each with the
float64 residual and a BiCGStab solve of the bordered Newton system, history commit.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  value = crack-increments/s of the mixed-precision solver
(float32 FFTs / Krylov, float64 residual and constraint), whole job over N GPUs (a batch of
independent RVEs per rank, advanced concurrently; weak scaling).  Also reported: operator-applies/s, the plain
float64 solver on the same workload, the operator apply's roofline, the float64 CPU oracle
on a bounded sample, an end-to-end figure through the public API with host buffers, SM
clocks during the timed region and the number of library kernel launches.
"""
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

import numpy as np  # noqa: E402

WORKLOAD = "composite512: 512x512 plane strain, RSA fibres r=12 at 40%, Ef/Em=10, nu 0.25/0.35, Gcf/Gcm=5, l=2, central notch 32, da=1"
METRIC = "crack-increments/s & operator-applies/s (% HBM roofline), batched vs plain FP64"
L2_BYTES = 129 * 1024 * 1024


def make_input(rank=0):
    from paper_2412_17445_gb300 import microstructure as ms
    return ms.fibre_composite(n=512, radius=12.0, fraction=0.4, notch_len=32,
                              seed=ms.SEED_BASE + 1 + 1000 * rank)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for i, nm in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def combine_ranks(torch, dist, t_local, units, applies, device):
    """Whole-job figures over the ranks: the slowest rank's timed seconds and the units
    (increments) and operator applies summed over all ranks.  No collective when dist is
    None (one process)."""
    if dist is None:
        return t_local, units, applies
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cnt = torch.tensor([float(units), float(applies)], device=device, dtype=torch.float64)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    return float(tt.item()), int(round(cnt[0].item())), int(round(cnt[1].item()))


def flush_l2(torch, buf):
    buf.add_(1.0)


def run_solver(torch, B, inp, precision, steps, warmup, flush, newton_tol=1e-8, krylov_tol=None):
    """One RVE alone on the current torch stream: start-up, W warm-up increments, K timed
    increments (CUDA events per step, L2 flushed between steps outside the events).  Returns
    the handle and a dict with times, the timed and warm-up records and the launches."""
    kt = krylov_tol if krylov_tol is not None else (1e-10 if precision == B.RVE_FP64 else 1e-2)
    g = B.RVE(inp, precision=precision, newton_tol=newton_tol, krylov_tol=kt)
    stream = torch.cuda.current_stream()
    g.set_stream(stream.cuda_stream)
    g.startup()
    warm = [g.crack_increment(1.0) for _ in range(warmup)]
    torch.cuda.synchronize()
    times, recs = [], []
    launches0 = g.kernel_launches()
    for _ in range(steps):
        flush_l2(torch, flush)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rec = g.crack_increment(1.0)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        recs.append(rec)
    launches = g.kernel_launches() - launches0
    return g, dict(times=times, recs=recs, warm=warm, launches=launches)


def apply_roofline(torch, B, g, inp, reps=50):
    """Operator apply timed alone (CUDA events on the apply's stream) at the current state."""
    n = g.n
    c = g.m + 1
    dt = torch.float32 if g.precision == B.RVE_MIXED else torch.float64
    g.linearize(B.RVE_CTRL_CRACK, 0.0)
    x = torch.randn(c * n, device="cuda", dtype=dt)
    y = torch.empty_like(x)
    xE = torch.zeros(1, device="cuda", dtype=torch.float64)
    yE = torch.zeros(1, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream()
    g.set_stream(stream.cuda_stream)
    for _ in range(5):
        g.apply_device(x.data_ptr(), xE.data_ptr(), y.data_ptr(), yE.data_ptr())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.apply_device(x.data_ptr(), xE.data_ptr(), y.data_ptr(), yE.data_ptr())
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    p = 4 if dt == torch.float32 else 8
    m = g.m
    # algorithmic bytes per voxel of one apply: p (6c + m + 2) (2D) / p (10c + m + 2) (3D)
    per_voxel = p * ((6 if g.dim == 2 else 10) * c + m + 2)
    return t, per_voxel * n


# DRAM bytes (read + write) of one grouped launch sequence of the 512^2 float32 apply over 4
# RVEs (k_xfwd_apply + k_col_fused2d + k_xinv_apply, blockIdx.y = RVE), summed from one ncu
# capture of the kernels whose sources hash to "sha" (the capture's command and per-kernel
# figures are kept with the other ncu summaries under profiles/); reported only while the
# sources still hash to it, null otherwise.
# GB300's float64 rate: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2070 MHz = 1.26 TFLOP/s
# (nominal 1.25), 1/64 of its float32 rate
FP64_TFLOPS = 1.25

APPLY_TRAFFIC = {"sha": "1a8f7543afd5cb90", "bytes": 116208384, "rves": 4}
APPLY_SOURCES = ["fft.cuh", "fft_passes.cuh", "rve_kern.cuh", "krylov_fin.cuh", "fft_inst_ct.cuh", "kernels_fft_512.cu"]


def apply_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in APPLY_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_17445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return APPLY_TRAFFIC["bytes"] if h.hexdigest()[:16] == APPLY_TRAFFIC["sha"] else None


def apply_grouped(torch, B, gs, reps=40):
    """Operator applies of len(gs) RVEs of one shape as single launches per pass
    (rve_apply_device_batch), the grouping the batched step runs its BiCGStab iterations
    in, timed with CUDA events on the launching stream.  Returns seconds per grouped
    launch sequence."""
    n = gs[0].n
    c = gs[0].m + 1
    st = torch.cuda.current_stream()
    for g in gs:
        g.set_stream(st.cuda_stream)
        g.linearize(B.RVE_CTRL_CRACK, 0.0)
    xs = [torch.randn(c * n, device="cuda", dtype=torch.float32) for _ in gs]
    xEs = [torch.zeros(1, device="cuda", dtype=torch.float64) for _ in gs]
    ys = [torch.empty_like(x) for x in xs]
    yEs = [torch.zeros(1, device="cuda", dtype=torch.float64) for _ in gs]
    args = ([x.data_ptr() for x in xs], [e.data_ptr() for e in xEs], [y.data_ptr() for y in ys],
            [e.data_ptr() for e in yEs])
    for _ in range(3):
        B.apply_device_batch(gs, *args)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        B.apply_device_batch(gs, *args)
    e1.record(st)
    e1.synchronize()
    for g in gs:
        g.set_stream(0)
    return e0.elapsed_time(e1) / 1e3 / reps


GOLDEN = os.path.join(ROOT, "tests", "golden", "composite512_crack.json")
ORACLE_COST = os.path.join(ROOT, "tests", "golden", "composite512_oracle_cost.json")


def _load_json(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def oracle_cost_per_increment():
    """The oracle's own work per crack increment of this workload at the float64 solver's
    benchmark tolerances, from its stored start-up + increments run (written by
    tests/golden/make_golden.py, which calls only the oracle): mean Newton and Krylov
    iterations per increment, the measured seconds per full increment and that host."""
    d = _load_json(ORACLE_COST)
    if not d or not d.get("rows"):
        return None
    rows = d["rows"]
    return {"newton": float(np.mean([r["newton"] for r in rows])), "krylov": float(np.mean([r["krylov"] for r in rows])),
            "increments": len(rows), "full_increment_s": [r["seconds"] for r in rows],
            "host": d.get("host"), "newton_tol": d.get("newton_tol"), "krylov_tol": d.get("krylov_tol")}


def cpu_sample(inp, budget_s=8.0, workers=None):
    """The float64 oracle as it stands on the host cores, on the 512^2 composite: seconds of
    one linearisation (constitutive update, residual) and of one Jacobian apply, each timed
    over a bounded number of calls (numpy.fft, or scipy.fft with `workers` threads)."""
    from oracle import fourier, solver
    from paper_2412_17445_gb300 import microstructure as ms
    fourier.set_fft_workers(workers)
    try:
        pb = solver.problem_from_input(inp)
        eps, E, phi, H = ms.random_state(inp, 3)
        dq = ms.random_direction(inp, 4)
        t0 = time.perf_counter()
        kl = 0
        while kl < 2 or (time.perf_counter() - t0 < 0.25 * budget_s and kl < 8):
            lin = solver.Linearization(pb, eps, E, phi, H)
            solver.residual(lin, solver.CRACK, lin.Gamma + 1.0)
            kl += 1
        t_lin = (time.perf_counter() - t0) / kl
        t0 = time.perf_counter()
        ka = 0
        while ka < 2 or time.perf_counter() - t0 < budget_s - kl * t_lin:
            solver.jacobian_apply(lin, dq, solver.CRACK)
            ka += 1
        t_app = (time.perf_counter() - t0) / ka
    finally:
        fourier.set_fft_workers(None)
    return {"linearize_s": t_lin, "apply_s": t_app, "linearizations": kl, "applies": ka,
            "seconds": kl * t_lin + ka * t_app, "workers": workers or 1}


def increment_seconds(sample, cost):
    """Seconds of one oracle increment: (Newton + 1) linearisations and 2 Krylov + 1 (the E
    column) applies per Newton iteration, with the oracle's own counts for this workload."""
    return (cost["newton"] + 1.0) * sample["linearize_s"] + (2.0 * cost["krylov"] + cost["newton"]) * sample["apply_s"]


def cpu_model():
    """CPU model of the host (lscpu's model name, else /proc/cpuinfo), with the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(inp):
    """cpu_baseline block of the JSON line: the oracle's increments/s on this host, single
    threaded and with scipy.fft on every core (the FFT is the only multi-threaded part)."""
    cost = oracle_cost_per_increment()
    one = cpu_sample(inp, 8.0, None)
    ncore = os.cpu_count() or 1
    many = cpu_sample(inp, 8.0, ncore)
    out = {"kind": "oracle", "cores": 1, "cpu": cpu_model(), "host_cores": ncore,
           "sample": "float64 oracle on the 512^2 composite: linearisations and Jacobian applies timed for about "
                     f"{one['seconds']:.0f} s (numpy, one thread); increments/s = 1 / ((Newton+1) t_lin + "
                     "(2 Krylov + Newton) t_apply) with the oracle's own Newton/Krylov counts per increment of this "
                     "workload (its stored run at Newton 1e-8, Krylov 1e-10)",
           "single_thread": one, "n_core": dict(many, cores=ncore, fft="scipy.fft workers=%d" % ncore)}
    if cost:
        out["value"] = 1.0 / increment_seconds(one, cost)
        out["unit"] = "crack-increments/s"
        out["n_core"]["value"] = 1.0 / increment_seconds(many, cost)
        out["oracle_counts"] = cost
    else:
        out["value"] = None
        out["unit"] = "crack-increments/s"
        out["note"] = "oracle cost file missing: no increment rate"
    return out


def golden_errors(recs_by_inc):
    """Relative errors of E and Sigma against the stored float64 oracle increments of the
    stored composite, for every increment that has a stored entry."""
    gold = _load_json(GOLDEN)
    if not gold:
        return None
    out = []
    for row in gold["rows"][1:]:
        r = recs_by_inc.get(row["inc"])
        if r is None:
            continue
        s = np.array(row["Sigma"])
        sig_o = np.array([s[0, 0], s[1, 1], math.sqrt(2.0) * s[0, 1]])
        out.append({"inc": row["inc"], "rel_E": abs(r["E"] - row["E"]) / abs(row["E"]),
                    "rel_sigma": float(np.max(np.abs(np.array(r["sigma"][:3]) - sig_o)) / np.max(np.abs(sig_o))),
                    "rel_gamma": abs(r["gamma"] - row["Gamma"]) / row["Gamma"]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16, help="RVEs advanced concurrently per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain float64 comparison")
    ap.add_argument("--no-extras", action="store_true", help="skip the long-run windows, porous, ragged and serving runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--porous-increments", type=int, default=25, help="increments of the 128^3 porous run in the extras")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-rate", type=float, default=0.4, help="Poisson arrival rate of the served stream (1/s)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2412_17445_gb300 import binding as B
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()
    flush = torch.zeros(2 * L2_BYTES // 4, device="cuda", dtype=torch.float32)
    nb = args.batch

    # ---- batched mixed-precision solver: nb independent 512^2 composites per rank ----
    inputs = [make_input(rank * nb + i) for i in range(nb)]
    gs = [B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8, krylov_tol=1e-2) for inp in inputs]
    for g in gs:
        g.startup()
    warm_out = []
    for _ in range(args.warmup):
        out_w, _ = B.batch_crack_increment(gs, [1.0] * nb)
        warm_out.append(out_w)
    launches0 = sum(g.kernel_launches() for g in gs)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    times, recs = [], []
    stream = torch.cuda.current_stream()
    for _ in range(args.steps):
        flush_l2(torch, flush)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out, st = B.batch_crack_increment(gs, [1.0] * nb)
        torch.cuda.synchronize()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        recs.append((out, st))
    clk = clocks.stop()
    launches = sum(g.kernel_launches() for g in gs) - launches0
    ok = sum(1 for out, st in recs for s_ in st if s_ == 0)
    applies = sum(o["applies"] for out, st in recs for o in out)
    t_batch, ok_all, applies_all = combine_ranks(torch, dist, sum(times), ok, applies, "cuda")
    inc_per_s = ok_all / t_batch
    applies_per_s = applies_all / t_batch

    # ---- single RVE, mixed: per-increment latency of one solve alone ----
    g1, one = run_solver(torch, B, make_input(rank), B.RVE_MIXED, max(1, args.steps), 1, flush)
    t_one = sum(one["times"]) / len(one["times"])

    # ---- operator apply alone (roofline of the dominant kernel chain) ----
    t_ap, bytes_ap = apply_roofline(torch, B, g1, make_input(rank))
    hbm, hbm_kind = peaks()
    achieved = bytes_ap / t_ap / 1e9
    # ---- the applies of one group of RVEs, one launch per pass (as in the batched step) ----
    n_grp = min(4, nb)
    t_grp = apply_grouped(torch, B, gs[:n_grp])
    # comparison point only: cuFFT (torch.fft) R2C + C2R of the same channels, no fused work
    from paper_2412_17445_gb300.apply_bench import cufft_roundtrip_us
    t_fft = cufft_roundtrip_us(torch, (512, 512), n_grp * (gs[0].m + 1), torch.float32, 40) * 1e-6
    cufft_cmp = {"cufft_roundtrip_us": t_fft * 1e6, "channels": n_grp * (gs[0].m + 1),
                 "grouped_apply_us": t_grp * 1e6, "apply_over_cufft": t_grp / t_fft,
                 "note": "torch.fft rfftn+irfftn of the group's float32 fields only; the apply also does the "
                         "projection, tangent, Helmholtz row and Krylov dots"}
    achieved_g = n_grp * bytes_ap / t_grp / 1e9

    # ---- end to end through the public API, every step: the states of all RVEs uploaded
    # from pinned host memory, the batched increment, the phase fields read back ----
    m, n = gs[0].m, gs[0].n
    host = []
    for g in gs:
        eps_h = torch.empty((m, n), dtype=torch.float64, pin_memory=True).numpy()
        phi_h = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        H_h = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        eps_h[:] = g.field(B.RVE_FIELD_EPS_T)
        phi_h[:] = g.field(B.RVE_FIELD_PHI)
        H_h[:] = g.field(B.RVE_FIELD_H)
        _, E0 = g.macro_stress()
        host.append((eps_h, phi_h, H_h, E0))
    taus = [o["tau"] for o in recs[-1][0]]
    e2e_times = []
    for _ in range(args.steps):
        flush_l2(torch, flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g, (eps_h, phi_h, H_h, E0), tau in zip(gs, host, taus):
            g.set_state(eps_h, phi_h, H_h, E0, tau)
        B.batch_crack_increment(gs, [1.0] * nb)
        for g in gs:
            g.field(B.RVE_FIELD_PHI)
        e2e_times.append(time.perf_counter() - t0)
    t_e2e, inc_e2e, _ = combine_ranks(torch, dist, sum(e2e_times), nb * args.steps, 0, "cuda")
    e2e = inc_e2e / t_e2e

    result = {
        "metric": METRIC, "value": inc_per_s, "unit": "crack-increments/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_batch / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed: f32 FFT/Krylov, f64 residual/constraint)",
        "data": "synthetic (seeded RSA fibre composites, 512^2, 40% fibres r=12)",
        "config": {"workload": WORKLOAD, "grid": [512, 512], "batch_per_gpu": nb,
                   "step": f"one crack increment of each of {nb} independent 512^2 composites (seeds differ): one host thread per RVE, BiCGStab chunks as grouped launches (up to 4 RVEs per launch)",
                   "newton_tol": 1e-8, "krylov_tol_mixed": 1e-2, "krylov_tol_fp64": 1e-10, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"independent RVEs, {nb} per GPU x{world} GPUs"},
        "increments_ok": ok_all, "increments_total": nb * args.steps * world,
        "operator_applies_per_s": applies_per_s,
        "applies_per_increment": applies_all / max(ok_all, 1),
        "single_rve_mixed": {"ms_per_increment": 1e3 * t_one, "increments_per_s": 1.0 / t_one,
                             "applies_per_increment": sum(r["applies"] for r in one["recs"]) / len(one["recs"])},
        "roofline": {"bound": "hbm", "achieved": achieved_g, "peak": hbm, "unit": "GB/s",
                     "frac": achieved_g / hbm,
                     "traffic": apply_traffic() if n_grp == APPLY_TRAFFIC["rves"] else None,
                     "kernel": f"operator apply of a group of {n_grp} 512^2 RVEs, one launch per pass as in the batched step "
                               "(x-forward+prologue, y fused projection, x-inverse+epilogue), float32",
                     "launch_us": t_grp * 1e6, "algorithmic_bytes": n_grp * bytes_ap, "peak_kind": hbm_kind},
        "cufft_comparison": cufft_cmp,
        "roofline_single_rve": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                "frac": achieved / hbm, "apply_us": t_ap * 1e6,
                                "kernel": "the same apply of one 512^2 RVE alone"},
        "e2e": {"value": e2e, "unit": "crack-increments/s", "h2d_bytes_per_step": nb * (m + 2) * n * 8,
                "d2h_bytes_per_step": nb * n * 8},
        "gpu_launches": launches,
        "clocks": clk,
    }
    # ---- error of the mixed results against the stored float64 oracle increments of the
    # stored composite (input 0 of rank 0: batch member 0 and the single-RVE run) ----
    if rank == 0:
        by_inc = {k + 1: o[0] for k, o in enumerate(warm_out + [r[0] for r in recs])}
        single = {k + 1: r for k, r in enumerate(one["warm"] + one["recs"])}
        result["mixed_vs_oracle"] = {
            "batched_member0": golden_errors(by_inc), "single_rve": golden_errors(single),
            "note": "relative errors of E, Sigma and Gamma against the float64 oracle (Newton/Krylov 1e-12) on the "
                    "increments it stores for this composite; target 1e-5"}
    if not args.no_fp64:
        # plain float64, one RVE at a time, on the same increments as the batched run (start-up,
        # the same W warm-up and K timed increments of input 0): at its own Krylov tolerance
        # 1e-10, and at the mixed run's tolerances (Newton 1e-8, Krylov 1e-2), so that
        # precision, tolerance and batching can be told apart
        torch.cuda.synchronize()
        fp = {}
        for tag, kt in (("krylov_1e-10", 1e-10), ("mixed_tolerances", 1e-2)):
            g64, f64 = run_solver(torch, B, make_input(rank), B.RVE_FP64, args.steps, args.warmup, flush,
                                  newton_tol=1e-8, krylov_tol=kt)
            t64 = sum(f64["times"])
            ap64 = sum(r["applies"] for r in f64["recs"])
            rate = len(f64["times"]) / t64
            entry = {"value": rate, "unit": "crack-increments/s", "newton_tol": 1e-8, "krylov_tol": kt,
                     "increments": [args.warmup + 1, args.warmup + args.steps],
                     "operator_applies_per_s": ap64 / t64, "applies_per_increment": ap64 / len(f64["times"]),
                     "newton_per_increment": float(np.mean([r["newton_iters"] for r in f64["recs"]])),
                     "cutbacks": int(sum(r["cutbacks"] for r in f64["recs"]))}
            if tag == "krylov_1e-10":
                t_ap64, bytes64 = apply_roofline(torch, B, g64, make_input(rank), reps=10)
                entry["apply_us"] = t_ap64 * 1e6
                # the float64 apply is bound by the FP64 pipe: flops per voxel from the model
                # 5 c log2(n) (forward + inverse FFTs) + 150 pointwise (2D), against the nominal
                # FP64 rate, and its algorithmic bytes against the measured HBM copy rate
                fpv = 5.0 * (g64.m + 1) * math.log2(g64.n) + (150.0 if g64.dim == 2 else 400.0)
                tf = fpv * g64.n / t_ap64 / 1e12
                entry["apply_roofline"] = {
                    "bound": "alu", "achieved": tf, "peak": FP64_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_TFLOPS,
                    "flops_per_voxel": fpv, "peak_kind": "nominal FP64 rate (152 SMs x 2 FP64 FMA/clock x 2070 MHz)",
                    "hbm_achieved_GBps": bytes64 / t_ap64 / 1e9, "hbm_frac": bytes64 / t_ap64 / 1e9 / hbm}
                if rank == 0:
                    entry["vs_oracle"] = golden_errors({k + 1: r for k, r in enumerate(f64["warm"] + f64["recs"])})
                # the batched member 0 against this run on the same increments
                pairs = [(o, f) for o, f in zip([r[0][0] for r in recs], f64["recs"])]
                if pairs:
                    entry["mixed_batched_vs_fp64"] = {
                        "max_rel_E": max(abs(a["E"] - b["E"]) / abs(b["E"]) for a, b in pairs),
                        "max_rel_sigma": max(max(abs(x - y) for x, y in zip(a["sigma"][:3], b["sigma"][:3]))
                                             / max(abs(y) for y in b["sigma"][:3]) for a, b in pairs)}
            fp[tag] = entry
            g64.close()
        result["fp64"] = dict(fp, note="plain float64 solver, one RVE at a time, same workload and increments as "
                                       "the batched run")
        result["batched_mixed_over_plain_fp64"] = inc_per_s / world / fp["krylov_1e-10"]["value"]
        result["batched_mixed_over_plain_fp64_same_tolerances"] = inc_per_s / world / fp["mixed_tolerances"]["value"]
    if rank == 0 and not args.no_extras:
        result["extras"] = extras(args)
    if rank == 0:
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(make_input(0))
        print(json.dumps(result))
    for g in gs:
        g.close()
    g1.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def extras(args):
    """Measurements beside the headline, each through the public API, wall clock around
    calls that return after their device work: windows of the 512^2 composite's long run
    (increments 6-25, 100-119, 280-299), the first increments of the 128^3 porous solid, one
    step of the ragged batch (40 2D + 24 3D RVEs) and a short served Poisson stream."""
    import types
    from paper_2412_17445_gb300 import workloads_bench as W
    out = {}
    t0 = time.perf_counter()
    out["composite512_windows"] = W.windows(types.SimpleNamespace(rve="composite512", window_increments=0))
    out["porous128_windows"] = W.windows(types.SimpleNamespace(rve="porous128", window_increments=args.porous_increments))
    out["ragged"] = W.ragged(types.SimpleNamespace(steps=1))
    out["serve"] = W.serve_fixed(types.SimpleNamespace(requests=args.serve_requests, rate=args.serve_rate,
                                                       max_active=16, fp64_sample=0))
    out["seconds"] = time.perf_counter() - t0
    return out


def reference_arm(args, world, rank):
    """The float64 CPU oracle as the reference arm, as it stands, on the host cores.  Each
    step is a bounded sample of one crack increment's work on the 512^2 composite (one
    linearisation and Jacobian applies, about 3 s); the step counts as the fraction of an
    increment that the oracle's own Newton/Krylov counts per increment give it."""
    if rank != 0:
        return
    cost = oracle_cost_per_increment()
    if cost is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's stored cost run of this workload is missing"}))
        return
    inp = make_input(0)
    steps = max(1, args.steps)
    units, secs = 0.0, 0.0
    for k in range(args.warmup + steps):
        smp = cpu_sample(inp, 3.0, None)
        if k >= args.warmup:
            units += smp["seconds"] / increment_seconds(smp, cost)
            secs += smp["seconds"]
    val = units / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "crack-increments/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded RSA fibre composite, 512^2, 40% fibres r=12)",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": val, "unit": "crack-increments/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "per step: one oracle linearisation + Jacobian applies for about 3 s (numpy, one "
                                   "thread), counted as that fraction of an increment under the oracle's own "
                                   f"{cost['newton']:.1f} Newton and {cost['krylov']:.0f} Krylov iterations per increment "
                                   "of this workload",
                         "oracle_counts": cost},
        "e2e": {"value": val, "unit": "crack-increments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
