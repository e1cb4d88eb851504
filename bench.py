"""Benchmark: FISTA iterations/s of the sub-sampled Fourier SAFT reconstruction.

One step = one complete reconstruction of one measurement vector: lambda by
the mu rule (one A^H apply and a max reduction on the device) followed by
`iters` FISTA iterations (two operator applies each), through the C ABI.
The operator (generator table) and its Lipschitz constant are built once per
geometry before the timed region, as the paper reuses sigma_max across
reconstructions; their setup times are reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload vol64]
  python bench.py --impl reference ...   # the FP64 CPU oracle, same workload

Multi-GPU (torchrun): independent replicas, one scene per rank (weak
scaling); no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

STRATEGY_NAMES = {"random": 0, "contiguous": 1, "equispaced": 2, "maximal": 3, "energy": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="vol64", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--strategy", default="random", choices=sorted(STRATEGY_NAMES))
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "tf32x3", "bf16", "bf16x2", "fp16", "fp16x2"],
                    help="arithmetic of the depth contractions (sfs_precision)")
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-study", action="store_true",
                    help="skip the BF16 / BF16X2 vs FP32 time-to-same-NMSE study")
    ap.add_argument("--batch-scenes", type=int, default=None,
                    help="scenes of the batched-serving measurement (0 skips it; default 16, "
                         "4 on the 64 x 64 x 256 workload)")
    ap.add_argument("--no-strategies", dest="strategies", action="store_false",
                    help="skip the random / contiguous / equispaced comparison on the 32 x 32 workload")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the run-time sweep of one apply over Nz = Nt and Nx = Ny")
    ap.add_argument("--no-backtracking", dest="backtracking", action="store_false",
                    help="skip the backtracking-FISTA measurement")
    ap.add_argument("--no-mixing", dest="mixing", action="store_false",
                    help="skip the Rademacher-mixing measurement")
    ap.add_argument("--crb-trials", type=int, default=50,
                    help="trials per random strategy of the Cramer-Rao study (0 skips it)")
    ap.add_argument("--serving-scenes", type=int, default=256,
                    help="scenes of the mixed-geometry serving measurement (0 skips it)")
    ap.add_argument("--learned-eval", type=int, default=1000,
                    help="held-out scenes of the learned-ISTA evaluation")
    ap.add_argument("--learned-steps", type=int, default=1250,
                    help="training steps of the learned unrolled ISTA measurement on the vol32 "
                         "workload (0 skips it)")
    ap.add_argument("--oracle-workers", type=int, default=0,
                    help="threads of the all-core FP64 oracle timing (0: every host core)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


# arithmetic of each contraction mode (the lateral FFTs and the FISTA update
# are c64 in every mode)
DTYPE_OF = {"fp32": "c64 (f32)",
            "tf32x3": "c64 (f32 state; contractions tf32 hi/lo x3 on tensor cores, f32 accumulate)",
            "bf16": "c64 (f32 state; contractions bf16 table x bf16 hi/lo spectra, f32 accumulate)",
            "bf16x2": "c64 (f32 state; contractions bf16 hi/lo table x bf16 hi/lo spectra, f32 accumulate)",
            "fp16": "c64 (f32 state; contractions fp16 table x fp16 hi/lo spectra, power-of-2 scaled, "
                    "f32 accumulate)",
            "fp16x2": "c64 (f32 state; contractions fp16 hi/lo table x fp16 hi/lo spectra, power-of-2 scaled, "
                      "f32 accumulate)"}
REDUCED = ("bf16", "bf16x2", "fp16", "fp16x2")


def precision_study(sfs, torch, geom, op, args, w, iters, y, L, x_true, flush, stream, oracle=None):
    """FISTA with the FP32 contractions against the 16-bit ones on the
    same scene, measurements, lambda rule and L: per mode the device time of
    one solve (L2 flushed first), the NMSE against the true scene, and the
    iterations and time a reduced-precision solve needs to reach the FP32
    solve's NMSE (first of K, 1.1 K, 1.25 K, 1.5 K, 2 K iterations within
    0.01 dB).  Errors are stated against the FP32 result of the same call
    and, when the FP64 oracle of the workload is given, against it: A x of
    the true scene, and the iterate after `oracle_iters` FISTA iterations
    (20, with the oracle's own lambda and the same L on both sides)."""
    xt = torch.from_numpy(x_true.astype(np.complex64)).cuda()
    ops = {}
    for mode in ("fp32",) + REDUCED:
        ops[mode] = op if args.precision == mode else sfs.Operator.from_indices(
            geom, op.idx, precision=sfs.PRECISION_NAMES[mode])

    def solve(o, k):
        x = torch.empty(o.shape_x, dtype=torch.complex64, device="cuda")
        o.fista(y, -w["mu"], L, k, x=x)  # warm (graph capture for k)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            o.fista(y, -w["mu"], L, k, x=x)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best, x.cpu().numpy().astype(np.complex128)

    def nmse_db(x):
        return float(10 * np.log10(np.linalg.norm(x - x_true) ** 2 / np.linalg.norm(x_true) ** 2))

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    ref = None
    if oracle is not None:
        O, oop, _, _ = oracle
        yh = y.cpu().numpy().astype(np.complex128)
        lam64 = O.lambda_from_mu(oop.apply_AH, yh, w["mu"])
        k64 = 20
        ax64 = oop.apply_A(x_true)
        x64 = O.fista(oop.apply_A, oop.apply_AH, yh, lam64, L, k64)
        ref = {"ax": ax64, "x": x64, "lam": lam64, "iters": k64}

    def vs_fp64(o):
        if ref is None:
            return {}
        axm = o.apply_A(xt).cpu().numpy().astype(np.complex128)
        xk = o.fista(y, ref["lam"], L, ref["iters"]).cpu().numpy().astype(np.complex128)
        return {"rel_err_Ax_vs_fp64": rel(axm, ref["ax"]),
                "rel_err_x%d_vs_fp64" % ref["iters"]: rel(xk, ref["x"]),
                "nmse_db_x%d" % ref["iters"]: nmse_db(xk)}

    ax32 = ops["fp32"].apply_A(xt).cpu().numpy().astype(np.complex128)
    t32, x32 = solve(ops["fp32"], iters)
    target = nmse_db(x32)
    out = {"reference": "fp32", "iters": iters, "target_nmse_db": target,
           "timing": "device time of one solve (lambda rule + iterations), best of 3, L2 flushed first",
           "modes": {"fp32": dict({"ms_per_solve": t32, "nmse_db": target,
                                   "table_bytes": ops["fp32"].info["table_bytes"]}, **vs_fp64(ops["fp32"]))}}
    if ref is not None:
        out["fp64_oracle"] = {"iters": ref["iters"], "nmse_db_x%d" % ref["iters"]: nmse_db(ref["x"]),
                              "note": "FP64 lateral-FFT oracle (Algorithm 2) on the host: A x of the true "
                                      "scene and FISTA with its own lambda (mu rule) and the same L"}
    for mode in REDUCED:
        o = ops[mode]
        axm = o.apply_A(xt).cpu().numpy().astype(np.complex128)
        tk, xk = solve(o, iters)
        rec = {"ms_per_solve": tk, "nmse_db": nmse_db(xk), "table_bytes": o.info["table_bytes"],
               "rel_err_Ax_vs_fp32": rel(axm, ax32), "rel_err_x_vs_fp32": rel(xk, x32)}
        rec.update(vs_fp64(o))
        reach = None
        for f in (1.0, 1.1, 1.25, 1.5, 2.0):
            k = int(math.ceil(f * iters))
            t, xk2 = (tk, xk) if k == iters else solve(o, k)
            if nmse_db(xk2) <= target + 0.01:
                reach = (k, t)
                break
        if reach is not None:
            rec.update({"iters_to_target": reach[0], "ms_to_target": reach[1],
                        "speedup_vs_fp32": t32 / reach[1]})
        else:
            rec.update({"iters_to_target": None, "ms_to_target": None, "speedup_vs_fp32": None})
        out["modes"][mode] = rec
    return out


def strategy_study(sfs, torch, args, flush, stream, seed):
    """The 32 x 32 x 128 workload's strategy comparison: random (per
    position), contiguous and equispaced bins, each set computed by the
    library's host selection and by the FP64 oracle's and compared bit for
    bit; per strategy FISTA it/s (device time of one solve, best of 3, L2
    flushed), the NMSE after the workload's iterations, the union U and
    the table bytes."""
    import oracle as O
    name = "vol32"
    out = {"workload": name, "strategies": {}}
    for strat in ("random", "contiguous", "equispaced"):
        ws = workload_setup(sfs, torch, name, strat, seed)
        w, op, y, L, x_true = ws["w"], ws["op"], ws["y"], ws["L"], ws["x_true"]
        go = O.Geometry(**synth.geometry_params(name))
        idx = O.select_indices(go, STRATEGY_NAMES[strat], w["M"], True, seed)
        x = torch.empty(op.shape_x, dtype=torch.complex64, device="cuda")
        op.fista(y, -w["mu"], L, w["iters"], x=x)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            flush.fill_(7)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            op.fista(y, -w["mu"], L, w["iters"], x=x)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        xh = x.cpu().numpy().astype(np.complex128)
        out["strategies"][strat] = {
            "identical_index_sets_cpu_gpu": bool(np.array_equal(op.idx, idx)),
            "U": op.info["U"], "table_bytes": op.info["table_bytes"], "iters": w["iters"],
            "ms_per_solve": best, "fista_it_per_s": w["iters"] / (best / 1e3),
            "nmse_db": float(10 * np.log10(np.linalg.norm(xh - x_true) ** 2 / np.linalg.norm(x_true) ** 2))}
    return out


def batched_study(sfs, torch, geom, op, args, w, iters, L, flush, stream, seed):
    """Serving pattern of a fixed acquisition setup: args.batch_scenes scenes
    (own scatterers and noise, same geometry and kept bins) solved by one
    sfs_fista_batched call, lambda by the mu rule per scene, the same L and
    iterations as the single-scene line.  Per precision: aggregate
    scene-iterations/s and the solve latency (every scene of a batch
    finishes with the batch) over 5 timed solves, L2 flushed before each."""
    B = args.batch_scenes
    ys = []
    for b in range(B):
        xt = torch.from_numpy(make_scene(w, seed + 100 + b).astype(np.complex64)).cuda()
        y0 = op.apply_A(xt).cpu().numpy().astype(np.complex128)
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, w["snr_db"])
        ys.append((y0 + sig * synth.unit_noise(y0.shape, seed=seed + 300 + b)).astype(np.complex64))
    y = torch.from_numpy(np.stack(ys)).cuda()
    out = {"scenes": B, "iters": iters, "unit": "scene-iterations/s",
           "timing": "device time of one batched solve (lambda rule + iterations), 5 solves, "
                     "L2 flushed before each; latency = solve time (all scenes finish together)",
           "modes": {}}
    for mode in ("fp32",) + REDUCED:
        o = op if args.precision == mode else sfs.Operator.from_indices(
            geom, op.idx, precision=sfs.PRECISION_NAMES[mode])
        x = torch.empty((B,) + o.shape_x, dtype=torch.complex64, device="cuda")
        o.fista_batched(y, -w["mu"], L, iters, x=x)  # workspace and graph capture
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            flush.fill_(2)
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            o.fista_batched(y, -w["mu"], L, iters, x=x)
            b2.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b2))
        ts.sort()
        out["modes"][mode] = {"value": B * iters / (statistics.mean(ts) / 1e3),
                              "latency_ms_p50": statistics.median(ts),
                              "latency_ms_p99": ts[-1],
                              # two plane launches; contractions per group of 4 scenes
                              # (16-bit) or per scene (FP32), forward and adjoint
                              "launches_per_iter": 2 + 2 * (B if mode == "fp32" else -(-B // 4))}
    return out


def backtracking_study(sfs, torch, op, w, iters, y, L, x_true, flush, stream):
    """sfs_fista_backtracking on the workload's scene (same iterations and mu
    rule) from the Frobenius lower bound L0 = ||A||_F^2 / N <= sigma_max^2,
    eta = 2: wall time of one solve (host-driven: one read per trial, L2
    flushed first, best of 2), the accepted L against the power-iteration
    L, and the NMSE beside the graph-replayed FISTA's with that L."""
    fro2, _ = op.frobenius()
    N = min(op.S * op.M, op.V)
    L0 = fro2 / N
    x = torch.empty(op.shape_x, dtype=torch.complex64, device="cuda")
    best, hist = None, None
    for _ in range(2):
        flush.fill_(6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, hist = op.fista_backtracking(y, -w["mu"], L0, 2.0, iters, x=x)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        best = t if best is None else min(best, t)

    def nmse_db(v):
        v = v.cpu().numpy().astype(np.complex128)
        return float(10 * np.log10(np.linalg.norm(v - x_true) ** 2 / np.linalg.norm(x_true) ** 2))

    xf = op.fista(y, -w["mu"], L, iters)
    return {"L0": L0, "eta": 2.0, "iters": iters, "ms_per_solve": best * 1e3,
            "fista_it_per_s": iters / best, "L_final": float(hist[-1]), "L_power_iteration": L,
            "backtracks": int(round(math.log(hist[-1] / L0, 2.0))), "nmse_db": nmse_db(x),
            "fista_nmse_db": nmse_db(xf),
            "timing": "wall time of one host-driven solve (one host read per trial), best of 2"}


def runtime_sweep(sfs, torch, flush, stream, seed):
    """Device time of one A and one A^H apply (FP32, best of 5 after one
    warm-up, L2 flushed before each) over Sec. V's run-time shapes: Nz = Nt
    at a 64 x 64 scan, and Nx = Ny at Nz = 5 (recipe synth.SWEEP)."""
    sw = synth.SWEEP

    def one(Nx, Nz, Nt):
        params = dict(synth.BASE, Nx=Nx, Ny=Nx, Nz=Nz, dz=0.15e-3, Nt=Nt, device=torch.cuda.current_device())
        g = sfs.Geometry(**params)
        M = max(1, Nt // 16)
        while True:
            try:
                op = sfs.Operator.select(g, sfs.SFS_SEL_RANDOM, M, True, seed)
                break
            except sfs.SfsError:
                if M == 1:
                    raise
                M = max(1, M // 2)
        xt = torch.from_numpy(synth.scene(op.shape_x, 10, "uniform", seed=seed).astype(np.complex64)).cuda()
        y = op.apply_A(xt)
        xo = op.apply_AH(y)
        torch.cuda.synchronize()
        ts = {"A": [], "AH": []}
        for _ in range(5):
            for key in ("A", "AH"):
                flush.fill_(5)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                if key == "A":
                    op.apply_A(xt, out=y)
                else:
                    op.apply_AH(y, out=xo)
                b.record(stream)
                torch.cuda.synchronize()
                ts[key].append(a.elapsed_time(b) * 1e3)
        return {"Nx": Nx, "Nz": Nz, "Nt": Nt, "M": M, "U": op.info["U"], "A_us": min(ts["A"]),
                "AH_us": min(ts["AH"])}

    out = {"unit": "us per apply (FP32, L2 flushed, best of 5)",
           "note": "the figure's 100 x 100 scan exceeds the 64 x 64 the lateral FFT engine holds; 64 x 64 stands in",
           "nz_eq_nt": [one(sw["nxy_at_nz"], n, n) for n in sw["nz_nt"]],
           "nx_eq_ny": [one(n, sw["nz"], sw["nt_for_nxy"]) for n in sw["nxy"]]}
    return out


def mixing_study(sfs, torch, args, flush, stream, seed):
    """The 32 x 32 x 128 workload measured through Rademacher-mixed A-scans
    (Phi_rnd,m,f: own xi_s and own random bins per position): band operator
    (the signed bins within 140 dB of the pulse peak, sfs_mixing_band, at
    every position) plus the mixing object; FISTA with the workload's
    iterations and mu rule, L by power iteration on A_mix.  Reports the
    device time of a solve (L2 flushed first, best of 3), FISTA it/s and
    the NMSE against the true scene, beside the unmixed solve's NMSE."""
    name = "vol32"
    ws = workload_setup(sfs, torch, name, "random", seed)
    w, geom, op, x_true = ws["w"], ws["geom"], ws["op"], ws["x_true"]
    iters, Nt = w["iters"], w["Nt"]
    xi = synth.rademacher((geom.S, Nt), seed=seed + 4242)
    mx = sfs.Mixing.create(geom, op.idx, xi)
    band = mx.band.idx[0]
    xt = torch.from_numpy(x_true.astype(np.complex64)).cuda()
    y0 = mx.apply_A(xt).cpu().numpy().astype(np.complex128)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, w["snr_db"])
    y = torch.from_numpy((y0 + sig * synth.unit_noise(y0.shape, seed=seed + 4343)).astype(np.complex64)).cuda()
    L, _ = mx.lipschitz(max_iter=300, rtol=1e-6, seed=seed, safety=1e-3)
    x = torch.empty(op.shape_x, dtype=torch.complex64, device="cuda")
    mx.fista(y, -w["mu"], L, iters, x=x)  # graph capture
    torch.cuda.synchronize()
    best = None
    for _ in range(3):
        flush.fill_(4)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mx.fista(y, -w["mu"], L, iters, x=x)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best = t if best is None else min(best, t)
    xh = x.cpu().numpy().astype(np.complex128)
    nmse = float(10 * np.log10(np.linalg.norm(xh - x_true) ** 2 / np.linalg.norm(x_true) ** 2))
    xu = op.fista(ws["y"], -w["mu"], ws["L"], iters).cpu().numpy().astype(np.complex128)
    nmse_u = float(10 * np.log10(np.linalg.norm(xu - x_true) ** 2 / np.linalg.norm(x_true) ** 2))
    return {"workload": name, "strategy": "Phi_rnd,m,f (xi_s and bins drawn per position)",
            "band_bins": int(band.size), "band_signed": [int(band[0]), int(band[-1])],
            "M": int(w["M"]), "iters": iters, "ms_per_solve": best, "fista_it_per_s": iters / (best / 1e3),
            "nmse_db": nmse, "unmixed_nmse_db": nmse_u, "L": L, "launches_per_iter": 6,
            "timing": "device time of one solve (lambda rule + iterations), best of 3, L2 flushed first"}


def crb_study(sfs, torch, args, seed):
    """Sec. VI's bound on locating one scatterer, per sampling strategy and
    kept bins per position n_f, relative to keeping every bin 0 .. Nt/2:
    C / C_full per coordinate (mean, min and max over args.crb_trials draws
    for the random strategies).  All index sets of a (strategy, n_f) pair go
    to one sfs_crb call; `gpu_s` is the wall time of those calls (FP64 sums
    on the GPU, host inversion, transfers included)."""
    cfg = synth.CRB
    g = sfs.Geometry(**dict(cfg["params"], device=torch.cuda.current_device()))
    kmax = cfg["params"]["Nt"] // 2
    full = np.tile(np.arange(kmax + 1, dtype=np.int32), (g.S, 1))
    c_full, _ = g.crb(full, cfg["pos"], 1.0, 0.0, 1.0)
    strategies = {"rnd": (sfs.SFS_SEL_RANDOM, False, True), "rnd_f": (sfs.SFS_SEL_RANDOM, True, True),
                  "max": (sfs.SFS_SEL_MAXIMAL, False, False), "nrg": (sfs.SFS_SEL_ENERGY, False, True),
                  "nrg_f": (sfs.SFS_SEL_ENERGY, True, True), "contiguous": (sfs.SFS_SEL_CONTIGUOUS, False, False),
                  "equispaced": (sfs.SFS_SEL_EQUISPACED, False, False)}
    out = {"setup": "50 x 50 scan, 0.5 mm, c 5920 m/s, fs 20 MHz, fc 3.2 MHz, 65 % bandwidth, theta 30 deg, "
                    "Nt 512, scatterer 33.3 mm below the centre",
           "n_f": list(cfg["n_f"]), "crb_full_m2": [float(v) for v in c_full[0]],
           "ratio": "C / C_full per coordinate (x, y, z)", "strategies": {}}
    t_gpu, n_sets = 0.0, 0
    for name, (st, per_pos, randomised) in strategies.items():
        rec = {"mean": [], "min": [], "max": []}
        for nf in cfg["n_f"]:
            T = args.crb_trials if randomised else 1
            sets = np.stack([g.select_indices(st, nf, per_pos, seed + 7919 * t)[0] for t in range(T)])
            t0 = time.perf_counter()
            c, _ = g.crb(sets, cfg["pos"], 1.0, 0.0, 1.0)
            t_gpu += time.perf_counter() - t0
            n_sets += T
            r = c / c_full[0]
            rec["mean"].append([float(v) for v in r.mean(axis=0)])
            rec["min"].append([float(v) for v in r.min(axis=0)])
            rec["max"].append([float(v) for v in r.max(axis=0)])
        out["strategies"][name] = rec
    out.update({"index_sets": n_sets, "gpu_s": t_gpu})
    return out


def serving_study(sfs, torch, args, flush, stream, seed):
    """args.serving_scenes scenes of the SERVING mix (36 geometry classes),
    one BF16 operator per class present (L by 60 power iterations), all
    solved by one sfs_fista_grouped call of 200 iterations (lambda by the mu
    rule per scene).  Reports aggregate scene-iterations/s over 3 timed
    solves (L2 flushed first) and the solve latency, which every scene
    shares; setup (tables, L) is timed apart."""
    sv = synth.SERVING
    classes = synth.serving_classes()
    draw = synth.serving_draw(args.serving_scenes, seed + 555)
    t0 = time.perf_counter()
    ops, ys, Ls, counts = [], [], [], []
    for c in sorted(set(draw.tolist())):
        n = int((draw == c).sum())
        g = sfs.Geometry(**dict(synth.serving_params(classes[c]), device=torch.cuda.current_device()))
        op = sfs.Operator.select(g, sfs.SFS_SEL_RANDOM, classes[c][2], True, seed + c,
                                 precision=sfs.SFS_PREC_BF16)
        op._geom = g
        L, _ = op.lipschitz(max_iter=60, rtol=1e-4, seed=seed, safety=1e-2)
        xt = torch.from_numpy(np.stack([synth.scene(op.shape_x, sv["n_scatter"], "uniform", seed=seed + 1000 * c + b)
                                        for b in range(n)]).astype(np.complex64)).cuda()
        y0 = op.apply_A_batched(xt).cpu().numpy().astype(np.complex128)
        yb = []
        for b in range(n):
            sig = synth.noise_scale(float(np.vdot(y0[b], y0[b]).real), y0[b].size, sv["snr_db"])
            yb.append(y0[b] + sig * synth.unit_noise(y0[b].shape, seed=seed + 2000 * c + b))
        ops.append(op)
        Ls.append(L)
        counts.append(n)
        ys.append(torch.from_numpy(np.stack(yb).astype(np.complex64)).cuda())
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    # tile of each class's batched contractions, by the library's autotuner
    t1 = time.perf_counter()
    tiles = {}
    for op_c, n in zip(ops, counts):
        nb, _ = op_c.autotune(n, reps=3)
        tiles[str(nb)] = tiles.get(str(nb), 0) + 1
    t_tune = time.perf_counter() - t1
    iters = sv["iters"]
    xs = sfs.fista_grouped(ops, ys, Ls, -0.05, iters)  # workspaces and graph capture
    torch.cuda.synchronize()
    ts, lat = [], []
    for _ in range(3):
        flush.fill_(3)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sfs.fista_grouped(ops, ys, Ls, -0.05, iters, xs=xs)
        b2.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b2))
        # each scene's latency: the completion of its class's loop in the graph
        for t_g, n in zip(sfs.grouped_times(len(ops)), counts):
            lat += [t_g] * n
    ts.sort()
    lat.sort()
    total = sum(counts)
    # the other priority orders of the grouped graph (same kernels, same
    # results): throughput and latency of 2 solves each
    orders = {}
    for name, order in (("largest_first", sfs.SFS_GROUPED_LARGEST_FIRST),
                        ("no_priority", sfs.SFS_GROUPED_NO_PRIORITY)):
        sfs.set_grouped_order(order)
        try:
            xo = sfs.fista_grouped(ops, ys, Ls, -0.05, iters)  # graph capture for this order
            torch.cuda.synchronize()
            to, lo = [], []
            for _ in range(2):
                flush.fill_(3)
                a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sfs.fista_grouped(ops, ys, Ls, -0.05, iters, xs=xo)
                b2.record(stream)
                torch.cuda.synchronize()
                to.append(a.elapsed_time(b2))
                for t_g, n in zip(sfs.grouped_times(len(ops)), counts):
                    lo += [t_g] * n
            same = all(torch.equal(p_, g_) for p_, g_ in zip(xo, xs))
        finally:
            sfs.set_grouped_order(sfs.SFS_GROUPED_CHEAPEST_FIRST)
        orders[name] = {"value": total * iters / (statistics.mean(to) / 1e3), "solve_ms": statistics.mean(to),
                        "latency_ms_p50": float(np.percentile(lo, 50)),
                        "latency_ms_p99": float(np.percentile(lo, 99)), "results_identical": same}
    # the same solve with the loops of all classes in one persistent kernel
    xg = [x.clone() for x in xs]
    t2 = time.perf_counter()
    policy, probe_ms = sfs.autotune_persistent(ops, ys, Ls, -0.05, probe_iters=10, reps=2)
    t_ptune = time.perf_counter() - t2
    xp = sfs.fista_persistent(ops, ys, Ls, -0.05, iters, nb_policy=policy)  # graph capture
    torch.cuda.synchronize()
    tp = []
    for _ in range(3):
        flush.fill_(3)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sfs.fista_persistent(ops, ys, Ls, -0.05, iters, xs=xp, nb_policy=policy)
        b2.record(stream)
        torch.cuda.synchronize()
        tp.append(a.elapsed_time(b2))
    step_ms = sfs.persistent_step_times()
    agree = max(float(torch.linalg.vector_norm(p_ - g_) / torch.linalg.vector_norm(g_))
                for pg, gg in zip(xp, xg) for p_, g_ in zip(pg, gg) if float(torch.linalg.vector_norm(g_)) > 0)
    persistent = {"value": total * iters / (statistics.mean(tp) / 1e3), "solve_ms": statistics.mean(tp),
                  "latency_ms_p50": statistics.mean(tp), "latency_ms_p99": statistics.mean(tp),
                  "max_rel_diff_vs_grouped": agree, "tile_policy": policy,
                  "step_ms_fwd_resid_adj_update": step_ms[:4],
                  "mean_cta_busy_ms_fwd_resid_adj_update": step_ms[4:],
                  "probe_ms_policies_0_1_2_4": probe_ms, "tile_tuning_s": t_ptune,
                  "note": "sfs_fista_persistent: one cooperative kernel runs all iterations of every class "
                          "(a grid barrier between the 4 steps of an iteration); every scene ends with the "
                          "solve. Before it, as in the grouped solve, the lambda rule per class and, in the "
                          "captured graph, 2 setup kernels per class"}
    return {"scenes": total, "classes": len(ops), "iters": iters, "precision": "bf16",
            "unit": "scene-iterations/s", "value": total * iters / (statistics.mean(ts) / 1e3),
            "solve_ms": statistics.mean(ts),
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_note": "per scene: from the start of the grouped call to the end of its class's loop "
                            "(event-record node in the graph), over 3 solves",
            "setup_s": t_setup, "autotune_s": t_tune, "tiles_chosen": tiles,
            "priority_order": "cheapest_first (sfs_set_grouped_order default)", "other_orders": orders,
            "persistent": persistent,
            "mix": "grids {16,32,48,64}^2, depths {64,128,256}, M {32,64,128}, 10 scatterers, 20 dB"}


def learned_study(sfs, torch, args, stream, seed):
    """Train the 16-layer unrolled ISTA (library kernels: forward, backward,
    Adam) for args.learned_steps steps of 8 fresh scenes of the LEARNED
    recipe (1250 steps: 10^4 scenes), then on args.learned_eval held-out
    scenes compare its NMSE and time with batched FISTA (same operator,
    lambda by the mu rule) at 4 .. 300 iterations: the first count of the
    ladder that reaches the network's NMSE, and its time."""
    from paper_2012_04534_gb300 import lista
    ws = workload_setup(sfs, torch, synth.LEARNED["workload"], "random", seed, args.precision
                        if args.precision in ("fp32", "bf16", "fp16") else "fp32")
    op, w, L = ws["op"], ws["w"], ws["L"]
    layers, B = synth.LEARNED["layers"], 8
    net = lista.LISTA(op, layers, B, L)
    rng = np.random.default_rng(seed + 4242)
    p = []
    for _ in range(layers):
        p.append(np.concatenate([[1.0, w["mu"]], 0.02 * rng.standard_normal(432), np.zeros(8),
                                 0.02 * rng.standard_normal(432), np.zeros(2)]))
    net.set_params(np.concatenate(p).astype(np.float32))

    def batch(base):
        xs, snrs = zip(*[synth.learned_draw(op.shape_x, base + b) for b in range(B)])
        xt = torch.from_numpy(np.stack(xs).astype(np.complex64)).cuda()
        y0 = op.apply_A_batched(xt).cpu().numpy().astype(np.complex128)
        ys = []
        for b in range(B):
            sig = synth.noise_scale(float(np.vdot(y0[b], y0[b]).real), y0[b].size, snrs[b])
            ys.append(y0[b] + sig * synth.unit_noise(y0[b].shape, seed=base + b + 99991))
        return torch.from_numpy(np.stack(ys).astype(np.complex64)).cuda(), xt

    steps = args.learned_steps
    t0 = time.perf_counter()
    for step in range(1, steps + 1):
        yb, xb = batch(seed * 1000003 + step * B)
        x = net.forward(yb)
        _, gx = net.nmse(x, xb)
        g = net.backward(gx)
        lr = 3e-3 * (0.5 * (1 + math.cos(math.pi * (step - 1) / steps)))
        net.adam(g, max(lr, 2e-5), step)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    evals = [batch(10 ** 9 + 97 * k) for k in range(max(1, args.learned_eval // B))]

    def timed(f):
        """Device time per evaluation batch of f(y) (after a warm call on the
        first batch, which also captures FISTA's graphs) and f's outputs."""
        f(evals[0][0])
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        outs = [f(y) for y, _ in evals]
        b2.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b2) / len(evals), outs

    def mean_nmse(xs):
        v = []
        for (_, xt), x in zip(evals, xs):
            num = ((x - xt).abs() ** 2).sum(dim=(1, 2, 3))
            den = (xt.abs() ** 2).sum(dim=(1, 2, 3))
            v += (num / den).tolist()
        return float(10 * np.log10(np.mean(v)))

    ms_lista, xs = timed(lambda y: net.forward(y))
    nmse_lista = mean_nmse(xs)
    ladder = []
    reach = None
    for K in (4, 8, 16, 32, 64, 128, 160, 192, 224, 256, 272, 288, 300):
        ms_k, xk = timed(lambda y, K=K: op.fista_batched(y, -w["mu"], L, K))
        nm = mean_nmse(xk)
        ladder.append({"iters": K, "nmse_db": nm, "ms_per_batch": ms_k})
        if reach is None and nm <= nmse_lista:
            reach = (K, ms_k)
    # the target: plain FP32 FISTA's NMSE after the workload's iterations
    target = ladder[-1]["nmse_db"]
    fista_to_target = next(r for r in ladder if r["nmse_db"] <= target + 0.01)

    def net_then_fista(y, K):
        x0 = net.forward(y)
        return op.fista_batched(y, -w["mu"], L, K, x=x0, warm_start=True) if K > 0 else x0

    warm = []
    warm_reach = None
    for K in (0, 8, 16, 32, 48, 64, 96, 128, 136, 144, 152, 160, 192, 224, 256, 300):
        ms_k, xk = timed(lambda y, K=K: net_then_fista(y, K))
        nm = mean_nmse(xk)
        warm.append({"fista_iters": K, "nmse_db": nm, "ms_per_batch": ms_k})
        if nm <= target + 0.01:
            warm_reach = (K, ms_k)
            break
    return {"layers": layers, "batch": B, "train_steps": steps, "train_scenes": steps * B,
            "train_s": t_train, "precision": op.info["precision"],
            "scenes": "1-20 scatterers, U(0.5,1) magnitudes, uniform phase, 10-30 dB SNR "
                      "(training scenes drawn fresh every step; %d held-out scenes)" % (len(evals) * B),
            "nmse_db": nmse_lista, "ms_per_batch": ms_lista,
            "fista": ladder,
            "fista_iters_to_same_nmse": None if reach is None else reach[0],
            "fista_ms_to_same_nmse": None if reach is None else reach[1],
            "speedup_vs_fista": None if reach is None else reach[1] / ms_lista,
            "target": {"what": "mean NMSE of plain FP32 FISTA after %d iterations (within 0.01 dB)"
                               % ladder[-1]["iters"], "nmse_db": target},
            "fista_to_target": {"iters": fista_to_target["iters"], "ms_per_batch": fista_to_target["ms_per_batch"]},
            "network_plus_fista": warm,
            "network_plus_fista_to_target": None if warm_reach is None else
            {"fista_iters": warm_reach[0], "ms_per_batch": warm_reach[1],
             "speedup_vs_fista": fista_to_target["ms_per_batch"] / warm_reach[1]}}


def workload_desc(name, w, strategy, iters):
    if w["Ny"] == 1:
        shape = "2-D line scan %d positions, %dx%d voxels" % (w["Nx"], w["Nx"], w["Nz"])
    else:
        shape = "3-D %dx%d scan, %dx%dx%d voxels" % (w["Nx"], w["Ny"], w["Nx"], w["Ny"], w["Nz"])
    return ("%s: %s, Nt=%d, M=%d %s bins per position, %d FISTA iterations, mu=%g, "
            "%g dB SNR" % (name, shape, w["Nt"], w["M"], strategy, iters, w["mu"], w["snr_db"]))


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle ---

def host_cores():
    return os.cpu_count() or 1


def mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def oracle_table_gb(name, w, strategy, seed):
    """Host memory of the FP64 oracle's generator table for a workload."""
    import oracle as O
    params = synth.geometry_params(name)
    go = O.Geometry(**params)
    idx = O.select_indices(go, STRATEGY_NAMES[strategy], w["M"], True, seed)
    U = np.unique(idx).size
    return U * w["Nz"] * (2 * w["Nx"] - 1) * (2 * w["Ny"] - 1) * 16 / 2 ** 30


def oracle_setup(name, w, strategy, seed, workers=1):
    """The FP64 lateral-FFT oracle of a workload (Algorithm 2) and its noisy
    measurements of the workload's scene: (O, operator, y, table build s)."""
    import oracle as O
    params = synth.geometry_params(name)
    go = O.Geometry(**params)
    idx = O.select_indices(go, STRATEGY_NAMES[strategy], w["M"], True, seed)
    t0 = time.perf_counter()
    op = O.LateralFFTOperator(go, idx, workers=workers)
    t_table = time.perf_counter() - t0
    x_true = make_scene(w, seed)
    y0 = op.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, w["snr_db"])
    y = y0 + sig * synth.unit_noise(y0.shape, seed=seed + 1)
    return O, op, y, t_table


def time_oracle_iterations(O, op, y, mu, seconds, workers=None):
    """FISTA iterations of the FP64 oracle for about `seconds` on `workers`
    threads (the operator's own count if None); returns (iterations/s,
    iterations done, threads actually used: CPU time / wall time)."""
    if workers is not None:
        op.workers = workers
    lam = O.lambda_from_mu(op.apply_AH, y, mu)
    L = 1.0e9  # step size does not change the work per iteration
    # one iteration first to size the sample
    t0 = time.perf_counter()
    O.fista(op.apply_A, op.apply_AH, y, lam, L, 1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-6)))
    c0, t0 = time.process_time(), time.perf_counter()
    O.fista(op.apply_A, op.apply_AH, y, lam, L, n)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return n / wall, n, max(1, round(cpu / wall))


def cpu_baseline_both(O, op, y, mu, seconds, cores):
    """The oracle as it stands, single-thread and on `cores` threads, each
    for about `seconds`: (all-core record, single-thread record)."""
    v1, n1, c1 = time_oracle_iterations(O, op, y, mu, seconds, workers=1)
    vn, nn, cn = time_oracle_iterations(O, op, y, mu, seconds, workers=cores)
    return (dict(value=vn, iters=nn, cores=cn, workers=cores),
            dict(value=v1, iters=n1, cores=c1, workers=1))


def make_scene(w, seed):
    shape = (w["Nz"], w["Ny"], w["Nx"])
    if w.get("n_scatter") is None:
        return synth.scene(shape, None, w["amp"], seed=seed, p_bernoulli=w["p_bernoulli"])
    return synth.scene(shape, w["n_scatter"], w["amp"], seed=seed)


# ------------------------------------------------------------------- main ---

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world):
    """The slowest rank's time: an all-reduce MAX over the process group (on
    the GPU with NCCL, on the CPU with gloo); ms itself for one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, iters, ms):
    """Whole-job FISTA iterations/s: every rank runs steps x iters (its own
    scene, weak scaling) within the slowest rank's time ms."""
    return world * steps * iters / (ms / 1e3)


def rank_seed(rank):
    """Seed of a rank's scene, noise, selection and power iteration."""
    return 1001 + 17 * rank


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle, as it stands, on rank 0, on
    every host core (its threads split independent planes and wavenumbers)."""
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    iters = args.iters or w["iters"]
    cores = args.oracle_workers or host_cores()
    need = oracle_table_gb(args.workload, w, args.strategy, 1001)
    if mem_available_gb() < 2.5 * need + 4:
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle's %.1f GB table does not fit "
                          "the host memory available (%.1f GB)" % (need, mem_available_gb())}), flush=True)
        return
    O, op, y, _ = oracle_setup(args.workload, w, args.strategy, seed=1001, workers=cores)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        time_oracle_iterations(O, op, y, w["mu"], per_step)
    vals, n_tot, threads, t_tot = [], 0, 1, 0.0
    for _ in range(args.steps):
        v, n, threads = time_oracle_iterations(O, op, y, w["mu"], per_step)
        vals.append(v)
        n_tot += n
        t_tot += n / v
    value = n_tot / t_tot
    line = {
        "impl": "reference", "metric": "FISTA iterations/s", "value": value,
        "unit": "it/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, w, args.strategy, iters)},
        "cpu_baseline": {"value": value, "unit": "it/s", "cores": threads, "kind": "oracle",
                         "sample": "%d FISTA iterations of the FP64 lateral-FFT oracle over "
                                   "%d steps, %d threads" % (n_tot, args.steps, cores)},
        "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Sources that define the contraction kernels or their launch shapes (the
# FP32, TF32X3 and 16-bit contractions, the plane data they read, their
# shared headers); a traffic record taken on other versions of these is stale.
CONTRACTION_SOURCES = ("sfs_kernels.cu", "sfs_tc.cu", "sfs_tc16.cu", "sfs_tc16_dev.cuh", "sfs_internal.h",
                       "sfs_launch.h", "sfs_async.cuh", "sfs_tcgen05.cuh", "sfs_fft.cuh", "sfs_planes.cuh")


def kernel_source_hash():
    """Hash of the contraction kernels' source files."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2012_04534_gb300", "csrc")
    for f in CONTRACTION_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, strategy, precision):
    """DRAM bytes per contraction launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "contract_traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    key = "%s/%s/%s" % (workload, strategy, precision)
    ent = rec.get(key)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent


def workload_setup(sfs, torch, name, strategy, seed, precision="fp32", lip_iters=500):
    """Operator, scene, noisy measurements (host and device) and L of a
    workload on the current device; setup times are returned apart."""
    w = synth.WORKLOADS[name]
    params = dict(synth.geometry_params(name), device=torch.cuda.current_device())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    geom = sfs.Geometry(**params)
    op = sfs.Operator.select(geom, STRATEGY_NAMES[strategy], w["M"], True, seed,
                             precision=sfs.PRECISION_NAMES[precision])
    op._geom = geom
    torch.cuda.synchronize()
    t_table = time.perf_counter() - t0
    x_true = make_scene(w, seed)
    xt = torch.from_numpy(x_true.astype(np.complex64)).cuda()
    y0 = op.apply_A(xt)
    torch.cuda.synchronize()
    y0h = y0.cpu().numpy().astype(np.complex128)
    sig = synth.noise_scale(float(np.vdot(y0h, y0h).real), y0h.size, w["snr_db"])
    y_host = (y0h + sig * synth.unit_noise(y0h.shape, seed=seed + 1)).astype(np.complex64)
    y = torch.from_numpy(y_host).cuda()
    t0 = time.perf_counter()
    L, _ = op.lipschitz(max_iter=lip_iters, rtol=1e-6, seed=seed, safety=1e-3)
    t_lip = time.perf_counter() - t0
    return dict(w=w, geom=geom, op=op, x_true=x_true, y=y, y_host=y_host, L=L,
                t_table=t_table, t_lip=t_lip)


def device_caps(torch, dev):
    """(SM count, L2 bytes) of the device, read from the driver."""
    p = torch.cuda.get_device_properties(dev)
    return int(p.multi_processor_count), int(getattr(p, "L2_cache_size", 0) or 0)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2012_04534_gb300 import build as sfs_build
    if rank == 0 or world == 1:
        sfs_build.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
        sfs_build.build()
    from paper_2012_04534_gb300 import sfs

    dev = local
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS[args.workload]
    iters = args.iters or w["iters"]
    seed = rank_seed(rank)
    n_sm, l2_bytes = device_caps(torch, dev)

    # ---- setup (outside the timed region) ----
    ws = workload_setup(sfs, torch, args.workload, args.strategy, seed, args.precision)
    geom, op, x_true, y, y_host, L = ws["geom"], ws["op"], ws["x_true"], ws["y"], ws["y_host"], ws["L"]
    t_table, t_lip = ws["t_table"], ws["t_lip"]
    info = op.info
    x = torch.empty(op.shape_x, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        # the iteration graph with event nodes around the kernels of <= 8
        # sampled iterations: the per-kernel times of the roofline come from
        # this same timed loop
        op.fista(y, -w["mu"], L, iters, x=x, time_kernels=True)

    def step_plain():
        op.fista(y, -w["mu"], L, iters, x=x)

    for _ in range(args.warmup):
        step()
        step_plain()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # L2 flush between timed steps: write a buffer larger than the L2
    flush = torch.empty(max(256 << 20, 2 * l2_bytes), dtype=torch.uint8, device="cuda")

    stage_acc = {"sum": np.zeros(4), "n": 0}

    def timed_steps(fn, stages=False):
        """Per-step CUDA events on the library's stream; the L2 flush runs
        between steps, outside the events.  Returns the summed step time [ms].
        With stages, the sampled per-kernel times of every step are added up
        (read after each step's end event, outside the timed span)."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
            if stages:
                evs[i][1].synchronize()
                ms4, n = op.stage_times()
                stage_acc["sum"] += np.asarray(ms4) * n
                stage_acc["n"] += n
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    # ---- timed region: device time, inputs resident ----
    clocks = ClockSampler(dev)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed work
    torch.cuda.nvtx.range_push("timed")
    ms = timed_steps(step, stages=True)
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, world)
    value = job_rate(world, args.steps, iters, ms)
    # per step: the lambda rule (scatter_fwd, adjoint contraction, inv_store),
    # set_thresholds, scatter_y_planes and the first fwd_planes, then four
    # kernels per iteration (the momentum table of a fresh start is reused)
    launches_per_step = 4 * iters + 6 if iters > 0 else 4
    stage_ms = (stage_acc["sum"] / max(1, stage_acc["n"])).tolist()

    # the same steps on the graph without event nodes, for comparison
    barrier()
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(timed_steps(step_plain), world)

    # ---- end to end through the public API with pinned host buffers ----
    y_pin = torch.from_numpy(y_host).pin_memory()
    x_pin = torch.empty(op.shape_x, dtype=torch.complex64).pin_memory()
    y_dev = torch.empty_like(y)

    def e2e_step():
        y_dev.copy_(y_pin, non_blocking=True)
        op.fista(y_dev, -w["mu"], L, iters, x=x)
        x_pin.copy_(x, non_blocking=True)

    barrier()
    torch.cuda.synchronize()
    ms_e2e = timed_steps(e2e_step)
    barrier()
    ms_e2e = max_over_ranks(ms_e2e, world)
    e2e = job_rate(world, args.steps, iters, ms_e2e)

    # ---- roofline of the dominant kernels, from the timed loop's event nodes ----
    fwd_ms, adj_ms = stage_ms[0], stage_ms[2]
    Nk, U, Nz, Ns = info["Nkappa"], info["U"], info["Nz"], info["Nslot"]
    # algorithmic bytes per launch: the folded table plus the spectra read and
    # written; algorithmic flops: one complex multiply-add (8 flops) per
    # (wavenumber, bin, depth)
    alg_bytes = info["table_bytes"] + 8 * Ns * (Nz + U)
    alg_flops = 8.0 * Nk * U * Nz
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(peaks_path) as fh:
            pk = json.load(fh)
        peak = float(pk["hbm_gbs"])
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        tc_peak = float(pk["bf16_tflops"])
        peak_src = "measured"
    except (OSError, ValueError, KeyError):
        peak, sm_max, tc_peak, peak_src = 6800.0, 2070.0, 1900.0, "fallback"
    # FP32 FMA issue peak: SMs x 128 lanes x 2 flops x max SM clock
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    avg_ms = 0.5 * (fwd_ms + adj_ms)
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    achieved_tf = alg_flops / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
    traffic = measured_traffic(args.workload, args.strategy, args.precision)
    hbm_frac, alu_frac = achieved / peak, achieved_tf / alu_peak
    in_l2 = l2_bytes > 0 and alg_bytes <= l2_bytes
    if not in_l2:
        # the table streams from HBM on every launch
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": hbm_frac, "peak_source": peak_src + " (HBM copy bandwidth)"}
    elif args.precision in ("fp32",):
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_frac,
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flops x %.0f MHz" % (n_sm, sm_max)}
    else:
        roof = {"bound": "tensor", "achieved": achieved_tf, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / tc_peak, "peak_source": peak_src + " (cuBLAS BF16 burst)"}
    roof.update({"traffic": None if traffic is None else traffic["bytes_per_launch"],
                 "kernel": "depth contraction (forward and adjoint, averaged)",
                 "table_location": "L2-resident" if in_l2 else "HBM (table larger than the %.0f MB L2)"
                                   % (l2_bytes / 1e6),
                 "alg_bytes_per_launch": alg_bytes, "alg_flops_per_launch": alg_flops,
                 "hbm_frac": hbm_frac, "alu_frac": alu_frac,
                 "fwd_ms": fwd_ms, "adj_ms": adj_ms, "iterations_timed": stage_acc["n"],
                 "timing": "event-record nodes around the kernels of <= 8 sampled iterations of each "
                           "timed step's graph; stages sum to the time of those iterations",
                 "iteration_stages_ms": {"contract_fwd": stage_ms[0], "resid_planes": stage_ms[1],
                                         "contract_adj": stage_ms[2], "update_planes": stage_ms[3]},
                 "iteration_ms": ms / args.steps / max(1, iters)})

    ran_here = rank == 0 and world == 1
    # ---- FP64 oracle of the workload (CPU baseline and precision study) ----
    oracle = None
    cores = args.oracle_workers or host_cores()
    if ran_here and not (args.no_cpu_baseline and args.no_precision_study):
        need = oracle_table_gb(args.workload, w, args.strategy, seed)
        if mem_available_gb() >= 2.5 * need + 4:
            oracle = oracle_setup(args.workload, w, args.strategy, seed, workers=cores)

    # ---- precision study: reduced-precision contractions vs FP32 and the
    # FP64 oracle, time to the FP32 solve's NMSE ----
    study = None
    if ran_here and not args.no_precision_study:
        study = precision_study(sfs, torch, geom, op, args, w, iters, y, L, x_true, flush, stream,
                                oracle=oracle)

    # ---- batched serving: scenes sharing the operator in one solve ----
    batched = None
    nbatch = args.batch_scenes if args.batch_scenes is not None else (4 if args.workload == "vol64" else 16)
    if ran_here and nbatch > 0:
        args.batch_scenes = nbatch
        batched = batched_study(sfs, torch, geom, op, args, w, iters, L, flush, stream, seed)

    # ---- random / contiguous / equispaced on the 32 x 32 workload ----
    strategies = None
    if ran_here and args.strategies:
        strategies = strategy_study(sfs, torch, args, flush, stream, seed)

    # ---- run time of one apply over the shapes of the paper's run-time figure ----
    sweep = None
    if ran_here and args.sweep:
        sweep = runtime_sweep(sfs, torch, flush, stream, seed)

    # ---- FISTA with backtracking on the same scene ----
    backtracking = None
    if ran_here and args.backtracking:
        backtracking = backtracking_study(sfs, torch, op, w, iters, y, L, x_true, flush, stream)

    # ---- Rademacher mixing (Phi_rnd,m) on the 32 x 32 workload ----
    mixing = None
    if ran_here and args.mixing:
        mixing = mixing_study(sfs, torch, args, flush, stream, seed)

    # ---- Cramer-Rao bound of one scatterer per strategy and n_f ----
    crb = None
    if ran_here and args.crb_trials > 0:
        crb = crb_study(sfs, torch, args, seed)

    # ---- serving mix: scenes of many geometries in one grouped graph launch ----
    serving = None
    if ran_here and args.serving_scenes > 0:
        serving = serving_study(sfs, torch, args, flush, stream, seed)

    # ---- learned unrolled ISTA vs FISTA, time to the same NMSE ----
    learned = None
    if ran_here and args.learned_steps > 0:
        learned = learned_study(sfs, torch, args, stream, seed)

    # ---- CPU baseline: the FP64 oracle, bounded sample, rank 0 only ----
    cpu = None
    if ran_here and not args.no_cpu_baseline:
        if oracle is None:
            cpu = {"value": None, "unit": "it/s", "cores": 0, "kind": "oracle",
                   "sample": "not run: the FP64 oracle's table does not fit the host memory available"}
        else:
            O, oop, oy, t_otab = oracle
            allc, one = cpu_baseline_both(O, oop, oy, w["mu"], args.cpu_seconds, cores)
            cpu = {"value": allc["value"], "unit": "it/s", "cores": allc["cores"], "kind": "oracle",
                   "sample": "%d FISTA iterations of the FP64 lateral-FFT oracle on the same workload, "
                             "%d threads (table build %.1f s excluded)" % (allc["iters"], cores, t_otab),
                   "single_thread": {"value": one["value"], "unit": "it/s", "cores": one["cores"],
                                     "sample": "%d FISTA iterations, 1 thread" % one["iters"]},
                   "host_cores": host_cores()}

    if rank == 0:
        line = {
            "metric": "FISTA iterations/s", "value": value, "unit": "it/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_OF[args.precision], "data": "synthetic",
            "config": {
                "workload": workload_desc(args.workload, w, args.strategy, iters),
                "precision": args.precision,
                "parallelism": "replicas" if world > 1 else "single GPU",
                "l2": "L2 flushed before every timed step (%d MB buffer write outside the "
                      "per-step events); generator table %.0f MB, L2 %.0f MB"
                      % (flush.numel() >> 20, info["table_bytes"] / 1e6, l2_bytes / 1e6),
                "U": U, "Nkappa": Nk, "Nslot": Ns, "orbit_slots": info["GS"], "Nz": Nz,
                "P": [info["Px"], info["Py"]], "sms": n_sm,
                "setup_s": {"table_build": round(t_table, 4), "lipschitz": round(t_lip, 4)},
                "L": L,
                "value_graph_without_event_nodes": job_rate(world, args.steps, iters, ms_plain),
            },
            "e2e": {"value": e2e, "unit": "it/s",
                    "h2d_bytes_per_step": int(y_host.nbytes),
                    "d2h_bytes_per_step": int(x_pin.numel() * 8)},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof,
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        for key, val in (("precision_study", study), ("batched", batched), ("strategies", strategies),
                         ("learned", learned), ("serving", serving), ("crb", crb), ("mixing", mixing),
                         ("runtime_sweep", sweep), ("backtracking", backtracking)):
            if val is not None:
                line[key] = val
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
