"""Measurements of the workloads beside the 512^2 headline: a 3D porous RVE, a ragged batch of
2D and 3D RVEs, a served Poisson stream of increment requests, the J-integral along a
crack-controlled path in a homogeneous panel, and energy against length control.

  python -m paper_2412_17445_gb300.workloads_bench porous128 [--increments 3]
  python -m paper_2412_17445_gb300.workloads_bench ragged [--steps 2]
  python -m paper_2412_17445_gb300.workloads_bench serve [--requests 32] [--loads 0.5,0.8,0.95]
  python -m paper_2412_17445_gb300.workloads_bench jint [--n 512] [--increments 3]
  python -m paper_2412_17445_gb300.workloads_bench energy512 [--increments 3]
  python -m paper_2412_17445_gb300.workloads_bench windows [--rve composite512|porous128] [--window-increments 0]

Each prints one JSON line.  Inputs are seeded synthetic microstructures
(paper_2412_17445_gb300.microstructure); timings are wall clock around calls that return
only after their device work has finished.
"""
import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_17445_gb300 import binding as B  # noqa: E402
from paper_2412_17445_gb300 import microstructure as ms  # noqa: E402

SEED = ms.SEED_BASE + 40


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def porous128(args):
    """128^3 porous solid (15 % spheres r = 8 as E = 1e-6 phase, penny notch r = 10), mixed
    precision with alpha = 0.9; the float64 GPU solver on the same increments for the error
    of the mixed result."""
    inp = ms.porous_solid(n=128, radius=8.0, porosity=0.15, notch_radius=10.0)
    out = {"workload": "porous128: 128^3, 15% spherical pores r=8 (E=1e-6), penny notch r=10, l=2, da=1",
           "voxels": int(np.prod(inp.shape))}
    res = {}
    for name, prec in (("mixed", B.RVE_MIXED), ("fp64", B.RVE_FP64)):
        k = args.increments if name == "mixed" else max(1, min(args.increments, args.fp64_increments))
        g = B.RVE(inp, precision=prec, newton_tol=1e-8, alpha=0.9)
        t0 = time.perf_counter()
        su = g.startup()
        t_su = time.perf_counter() - t0
        recs, times = [], []
        for _ in range(k):
            t0 = time.perf_counter()
            try:
                r = g.crack_increment(1.0)
            except B.RVEError as e:
                recs.append({"error": str(e)})
                break
            times.append(time.perf_counter() - t0)
            recs.append(r)
        g.close()
        ok = [r for r in recs if "error" not in r]
        res[name] = ok
        out[name] = {"startup_s": t_su, "startup_E": su.get("E"), "increments": len(ok),
                     "failed": len(recs) - len(ok),
                     "s_per_increment": float(np.mean(times)) if times else None,
                     "increments_per_s": len(times) / sum(times) if times else 0.0,
                     "applies_per_increment": float(np.mean([r["applies"] for r in ok])) if ok else None,
                     "newton_per_increment": float(np.mean([r["newton_iters"] for r in ok])) if ok else None,
                     "E": [r["E"] for r in ok]}
        if len(recs) > len(ok):
            out[name]["error"] = recs[-1]["error"]
    m = min(len(res["mixed"]), len(res["fp64"]))
    if m:
        out["mixed_vs_fp64"] = {
            "increments_compared": m,
            "max_rel_E": max(_rel(res["mixed"][i]["E"], res["fp64"][i]["E"]) for i in range(m)),
            "max_rel_sigma_yy": max(_rel(res["mixed"][i]["sigma"][1], res["fp64"][i]["sigma"][1]) for i in range(m))}
        if out["fp64"]["s_per_increment"] and out["mixed"]["s_per_increment"]:
            out["mixed_over_fp64_speed"] = out["fp64"]["s_per_increment"] / out["mixed"]["s_per_increment"]
    return out


def _ragged_inputs(n2=40, n3=24, seed=SEED):
    """40 2D grids with sides from {128, 192, 256, 384, 512} per axis and 24 3D grids with
    sides from {32, 48, 64, 96} per axis; fibre composite or porous solid by seed."""
    rng = np.random.default_rng(seed)
    s2, s3 = [128, 192, 256, 384, 512], [32, 48, 64, 96]
    inps = []
    for i in range(n2):
        ny, nx = (int(v) for v in rng.choice(s2, 2))
        if rng.random() < 0.5:
            inps.append(ms.fibre_composite(n=nx, ny=ny, radius=12.0, fraction=0.4, notch_len=min(32, nx // 4),
                                           seed=seed + 100 + i))
        else:
            inps.append(ms.homogeneous_panel(nx, notch_len=nx // 8) if nx == ny else
                        ms.fibre_composite(n=nx, ny=ny, radius=12.0, fraction=0.2, notch_len=min(32, nx // 4),
                                           seed=seed + 100 + i))
    for i in range(n3):
        shape = tuple(int(v) for v in rng.choice(s3, 3))
        inps.append(ms.porous_solid(shape=shape, radius=4.0, porosity=0.1, notch_radius=min(shape) / 6.0,
                                    seed=seed + 200 + i, E_pore=1e-3))
    return inps


def ragged(args):
    inps = _ragged_inputs()
    gs = [B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8) for inp in inps]
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        list(ex.map(lambda g: g.startup(), gs))
    vox = np.array([int(np.prod(inp.shape)) for inp in inps])
    out, st = B.batch_crack_increment(gs, [1.0] * len(gs))  # warm-up (and tile tuning)
    times, oks, applies = [], 0, 0
    prof = getattr(args, "profile_step", False)
    for _ in range(args.steps):
        if prof:  # the timed steps between cudaProfilerStart / Stop (ncu --profile-from-start off)
            import torch
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        t0 = time.perf_counter()
        out, st = B.batch_crack_increment(gs, [1.0] * len(gs))
        times.append(time.perf_counter() - t0)
        if prof:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        oks += sum(1 for s in st if s == 0)
        applies += sum(o["applies"] for o, s in zip(out, st) if s == 0)
    for g in gs:
        g.close()
    t = sum(times)
    return {
        "workload": "ragged: 40 2D (sides 128-512 per axis) + 24 3D (sides 32-96 per axis) RVEs, mixed, one increment each per step",
        "rves": len(gs), "voxels_total": int(vox.sum()), "steps": args.steps,
        "s_per_step": t / args.steps, "increments_per_s": oks / t,
        "voxel_increments_per_s": float(vox.sum()) * args.steps / t,
        "increments_ok": oks, "increments_total": len(gs) * args.steps,
        "applies_per_increment": applies / max(oks, 1)}


def _serve_requests(n, seed=SEED + 1):
    """Requests: 2D sides {256, 384, 512, 768, 1024}, 3D sides {64, 96, 128}, composite or
    porous, da in {1, 2, 3, 4}, one increment after start-up."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        da = float(rng.integers(1, 5))
        if rng.random() < 0.75:
            nx = int(rng.choice([256, 384, 512, 768, 1024]))
            inp = ms.fibre_composite(n=nx, radius=12.0, fraction=0.4, notch_len=32, seed=seed + 10 + i)
        else:
            nn = int(rng.choice([64, 96, 128]))
            inp = ms.porous_solid(n=nn, radius=6.0, porosity=0.1, notch_radius=nn / 8.0, seed=seed + 10 + i,
                                  E_pore=1e-3)
        reqs.append((inp, da))
    return reqs


def _run_server(reqs, arrivals, budget, max_active, precision):
    s = B.Server(hbm_budget_bytes=budget, max_active=max_active)
    t0 = time.perf_counter()
    ids = []
    for (inp, da), ta in zip(reqs, arrivals):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(s.submit(inp, n_increments=1, da=da, precision=precision, newton_tol=1e-8))
    s.drain()
    wall = time.perf_counter() - t0
    res = s.poll(max_results=4096)
    s.close()
    lat = np.array([r["t_end"] - r["t_submit"] for r in res])
    ok = sum(1 for r in res if r["status"] == 0)
    return dict(wall_s=wall, completed=ok, failed=len(res) - ok, requests_per_s=ok / wall,
                p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)))


def serve(args):
    reqs = _serve_requests(args.requests)
    budget = 150 << 30
    # capacity: every request queued at t = 0 (closed loop)
    cap = _run_server(reqs, [0.0] * len(reqs), budget, args.max_active, B.RVE_MIXED)
    loads = [float(x) for x in args.loads.split(",")]
    by_load = []
    for load in loads:
        rate = load * cap["requests_per_s"]
        rng = np.random.default_rng(SEED + 2)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        r = _run_server(reqs, list(arrivals), budget, args.max_active, B.RVE_MIXED)
        r.update(load=load, arrival_rate_per_s=rate)
        by_load.append(r)
    # plain float64 solver one request at a time on a sample of the same requests
    k = min(args.fp64_sample, len(reqs))
    t0 = time.perf_counter()
    for inp, da in reqs[:k]:
        g = B.RVE(inp, precision=B.RVE_FP64, newton_tol=1e-8)
        g.startup()
        g.crack_increment(da)
        g.close()
    t64 = (time.perf_counter() - t0) / k
    return {
        "workload": "serve: Poisson stream, 2D 256-1024 composites (75%) / 3D 64-128 porous (25%), da 1-4, "
                    "start-up + 1 increment per request, HBM budget 150 GB, mixed",
        "requests": len(reqs), "capacity": cap, "open_loop": by_load,
        "fp64_one_at_a_time": {"s_per_request": t64, "requests_per_s": 1.0 / t64, "sample": k},
        "served_over_fp64": [r["requests_per_s"] / (1.0 / t64) for r in by_load]}


def serve_fixed(args):
    """The served stream at one fixed Poisson arrival rate (args.rate requests/s; no capacity
    run): the same request mix as `serve`, p50/p99 latency from submission to completion."""
    reqs = _serve_requests(args.requests)
    rng = np.random.default_rng(SEED + 2)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, len(reqs)))
    r = _run_server(reqs, list(arrivals), 150 << 30, args.max_active, B.RVE_MIXED)
    r.update(workload="serve: Poisson stream, 2D 256-1024 composites (75%) / 3D 64-128 porous (25%), da 1-4, "
                      "start-up + 1 increment per request, HBM budget 150 GB, mixed",
             requests=len(reqs), arrival_rate_per_s=args.rate)
    return r


def jint(args):
    """n^2 homogeneous panel (notch n/8, l = 2), mixed precision: crack-length increments
    (Delta a = 1) with the J-integral (rve_j_integral) on square contours of half-size 8, 16
    and 32 around the tip after each; wall time of one rve_j_integral call (it blocks)."""
    n = args.n
    inp = ms.homogeneous_panel(n, notch_len=n // 8)
    Gc = float(inp.Gc[0])
    g = B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8)
    g.startup()
    rows, t_j = [], []
    for _ in range(args.increments):
        r = g.crack_increment(1.0)
        phi = g.field(B.RVE_FIELD_PHI).reshape(n, n)
        tip = int(np.max(np.nonzero(phi[n // 2, : 3 * n // 4] > 0.5)[0]))
        Js = []
        for d in (8, 16, 32):
            box = (tip - d, n // 2 - d, tip + d, n // 2 + d)
            t0 = time.perf_counter()
            Js.append(g.j_integral(box))
            t_j.append(time.perf_counter() - t0)
        rows.append({"E": r["E"], "tip_x": tip, "J_over_Gc": [J / Gc for J in Js],
                     "spread": (max(Js) - min(Js)) / max(abs(J) for J in Js)})
    g.close()
    return {
        "workload": f"jint: {n}^2 homogeneous panel, notch {n // 8}, l=2, da=1, mixed; J on contours of half-size 8/16/32",
        "increments": rows, "j_call_ms": 1e3 * float(np.median(t_j)), "j_calls": len(t_j)}


def energy512(args):
    """512^2 fibre composite (the headline RVE), mixed precision: crack-controlled increments
    under length control (da = 1 voxel) and under energy control (Eq. SystemDisc,
    d tau = G_c of the matrix per increment), same start-up; time per increment and Krylov
    work of each, and the dissipated-energy constraint's share of a Newton iteration."""
    inp = ms.fibre_composite(n=512)
    Gm = float(inp.Gc[0])
    out = {"workload": "energy512: 512^2 composite (r=12, vf=0.4, Gc_f/Gc_m=5), mixed; length control da=1 vs "
                       "energy control dtau=Gc_m",
           "increments": args.increments}
    for name, c, da in (("length", B.RVE_CONSTRAINT_LENGTH, 1.0), ("energy", B.RVE_CONSTRAINT_ENERGY, Gm)):
        g = B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8, constraint=c)
        su = g.startup()
        recs, times = [], []
        for _ in range(args.increments):
            t0 = time.perf_counter()
            recs.append(g.crack_increment(da))
            times.append(time.perf_counter() - t0)
        g.close()
        out[name] = {"startup_tau": su["tau"], "s_per_increment": float(np.mean(times)),
                     "applies_per_increment": float(np.mean([r["applies"] for r in recs])),
                     "newton_per_increment": float(np.mean([r["newton_iters"] for r in recs])),
                     "E": [r["E"] for r in recs], "gamma": [r["gamma"] for r in recs],
                     "tau": [r["tau"] for r in recs]}
    return out


def _window_stats(recs, times, lo, hi):
    """Increments lo..hi (1-based, inclusive) of a run: time, Newton / Krylov work, cut-backs."""
    sel = [(r, t) for k, (r, t) in enumerate(zip(recs, times), start=1) if lo <= k <= hi and r is not None]
    if not sel:
        return None
    rs, ts = [r for r, _ in sel], [t for _, t in sel]
    return {"increments": [lo, hi], "done": len(rs), "s_per_increment": float(np.mean(ts)),
            "increments_per_s": len(ts) / sum(ts),
            "newton_per_increment": float(np.mean([r["newton_iters"] for r in rs])),
            "krylov_per_increment": float(np.mean([r["krylov_iters"] for r in rs])),
            "applies_per_increment": float(np.mean([r["applies"] for r in rs])),
            "cutbacks": int(sum(r["cutbacks"] for r in rs)),
            "float64_fallbacks": int(sum(r.get("fallbacks", 0) for r in rs)),
            "E": [rs[0]["E"], rs[-1]["E"]], "gamma": [rs[0]["gamma"], rs[-1]["gamma"]]}


def windows(args):
    """One RVE of a long crack-controlled run (mixed precision, Newton 1e-8, Krylov 1e-2),
    every increment timed on the wall clock (each call returns after its device work):
    the 512^2 composite of the headline (300 increments; windows 6-25, 100-119, 280-299) or
    the 128^3 porous solid (alpha = 0.9, 150 increments; windows 6-25, 70-89, 131-150).
    A failed increment ends the run (the record says where)."""
    if args.rve == "composite512":
        inp = ms.fibre_composite(n=512, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 1)
        total, wins, alpha = 300, [(6, 25), (100, 119), (280, 299)], 1.0
        name = "composite512: 512^2 fibre composite of the headline, da=1, 300 increments"
    else:
        inp = ms.porous_solid(n=128, radius=8.0, porosity=0.15, notch_radius=10.0)
        total, wins, alpha = 150, [(6, 25), (70, 89), (131, 150)], 0.9
        name = "porous128: 128^3, 15% spherical pores r=8 (E=1e-6), penny notch r=10, alpha=0.9, da=1, 150 increments"
    cap = getattr(args, "window_increments", 0)
    total = min(total, cap) if cap > 0 else total
    g = B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8, krylov_tol=1e-2, alpha=alpha)
    t0 = time.perf_counter()
    g.startup()
    t_su = time.perf_counter() - t0
    recs, times, err = [], [], None
    for k in range(total):
        t0 = time.perf_counter()
        try:
            recs.append(g.crack_increment(1.0))
        except B.RVEError as e:
            err = f"increment {k + 1}: {e}"
            break
        times.append(time.perf_counter() - t0)
    g.close()
    return {"workload": name, "precision": "mixed", "startup_s": t_su, "increments_done": len(recs),
            "float64_fallbacks": int(sum(r.get("fallbacks", 0) for r in recs)),
            "s_per_increment_all": float(sum(times) / max(len(times), 1)),
            "increments_planned": total, "error": err, "seconds": float(sum(times)),
            "windows": [w for w in (_window_stats(recs, times, lo, hi) for lo, hi in wins) if w is not None],
            "E_first_last": [recs[0]["E"], recs[-1]["E"]] if recs else None,
            "gamma_last": recs[-1]["gamma"] if recs else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["porous128", "ragged", "serve", "serve_fixed", "jint", "energy512", "windows"])
    ap.add_argument("--rate", type=float, default=0.4, help="serve_fixed: Poisson arrival rate (1/s)")
    ap.add_argument("--rve", default="composite512", choices=["composite512", "porous128"])
    ap.add_argument("--window-increments", type=int, default=0, help="windows: stop after this many (0: all)")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--increments", type=int, default=3)
    ap.add_argument("--fp64-increments", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--profile-step", action="store_true",
                    help="ragged: bracket the timed steps with cudaProfilerStart / Stop")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--loads", default="0.8", help="arrival rates as fractions of the capacity, comma-separated")
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--fp64-sample", type=int, default=4)
    args = ap.parse_args()
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()
    fn = {"porous128": porous128, "ragged": ragged, "serve": serve, "serve_fixed": serve_fixed, "jint": jint,
          "energy512": energy512, "windows": windows}[args.which]
    print(json.dumps(fn(args)))


if __name__ == "__main__":
    main()
