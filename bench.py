#!/usr/bin/env python3
"""Benchmark of the GB300 J/K build (one JSON line on stdout).

A step is one pass of the J/K hot path over one synthetic molecule: the
screening and work-list pass, the ERI + J/K digestion kernels of both
precision bands, the spherical transforms and the energy E_JK
(adft_jk_energy), with the basis (pairs and Schwarz bounds) built once before
timing, as in an SCF loop.  The metric is screened shell quartets per second
of the mixed-precision build (--precision mixed: FP64 band in native FP64,
FP32 band in FP32) on the 2,064-function molecule (the "~2k basis functions"
point); the plain FP64 build of the same molecule is timed after it, and the
60-atom molecule's mixed and FP64 builds are reported beside it.  Launch
shapes are autotuned per class pair on the 60-atom molecule of the same
recipe and installed before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--precision fp64|mixed] [--split S] [--grad] [--impl reference]

With N ranks (torchrun, one GPU each) the ranks share one molecule's build:
rank 0 assigns the (band, class pair) launches to ranks by their autotuned
times and broadcasts the partition, each rank evaluates its class pairs, and
one sum all-reduce of the partial energy per step (of J and K in the
end-to-end measurement) is the exchange; the value is one build's screened
quartets over the slowest rank's time (strong scaling).  batch256 shards
whole molecules across ranks instead.

--impl reference times the CPU oracle (the plain FP64 reference written from
the paper's definitions) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "J+K build sec & screened quartets/s at ~2k basis fns; mixed vs FP64 at 1e-6 Eh"
UNIT = "screened quartets/s"
WORKLOADS = {
    "c240": "96 heavy (3s2p1d) + 144 H (2s1p) atoms, 1-6 primitives, exponents 0.1-5e3, "
            "2064 spherical functions, thresh 1e-10, mixed FP32/FP64 (the ~2k-function point)",
    "c120": "48 heavy (4s3p2d1f) + 72 H (3s2p1d) atoms, 1-8 primitives, exponents 0.05-1e4, "
            "2448 spherical functions, thresh 1e-12, split 1e-5, mixed FP32/FP64",
    "c200": "80 heavy (4s3p2d1f) + 120 H (3s2p1d) atoms, 1-8 primitives, exponents 0.05-1e4, "
            "4080 spherical functions, thresh 1e-12, split 1e-5, mixed FP32/FP64",
    "c60": "24 heavy (3s2p1d) + 36 H (2s1p) atoms, 1-6 primitives, exponents 0.1-5e3, "
           "516 spherical functions, thresh 1e-10, mixed FP32/FP64",
    "small": "3 heavy (3s2p1d) + 5 H (2s1p) atoms, 1-6 primitives, exponents 0.1-5e3, "
             "67 spherical functions, thresh 1e-10, split 1e-5, mixed FP32/FP64 (profiling case)",
    "batch256": "256 molecules of 10-40 atoms (40 % heavy, 3s2p1d / 2s1p, 1-6 primitives), 86-344 "
                "spherical functions each; J, K and E (and with --grad the nuclear gradient) of every "
                "molecule in one batched, graph-captured call per step; thresh 1e-10, split 1e-5, "
                "mixed FP32/FP64",
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank, int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload(name):
    from paper_2406_11185_gb300 import synth
    mol, opt = synth.config(name)
    nocc = synth.default_nocc(mol, opt["nocc"])
    D = synth.make_density(mol, nocc, opt["dseed"])
    return mol, opt, D


def cpu_oracle_rate(mol, opt, D, budget_s=15.0, seed=7, nthreads=None, growth=1.6):
    """Oracle quartets/s on a bounded sample of the workload: the oracle's
    whole J/K (Schwarz bounds + screened scatter sum) over a random subset of
    the molecule's shells (all atoms kept), grown until it takes about
    budget_s / 4 or more; on all host cores, or on nthreads of them."""
    import oracle
    from paper_2406_11185_gb300 import synth
    rng = np.random.default_rng(seed)
    order = rng.permutation(mol.nshell)
    offs = np.cumsum([0] + [2 * l + 1 for _, l, _, _ in mol.shells])
    k = 12
    spent = 0.0
    while True:
        pick = np.sort(order[:k])
        sub = synth.Molecule(mol.atoms, mol.heavy, [mol.shells[i] for i in pick], mol.spherical)
        idx = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in pick])
        Ds = np.ascontiguousarray(D[np.ix_(idx, idx)])
        t = time.time()
        _, _, kept = oracle.jk(sub, Ds, opt["thresh"], return_kept=True, nthreads=nthreads)
        dt = time.time() - t
        spent += dt
        if dt > budget_s / 4 or k >= mol.nshell or spent > budget_s:
            break
        k_next = min(mol.nshell, int(k * growth) + 1)
        if spent + dt * (k_next / k) ** 4 > 2.0 * budget_s:  # the work grows about as k^4
            break
        k = k_next
    cores = os.cpu_count() if nthreads is None else int(nthreads)
    how = "all host cores via OpenMP" if nthreads is None else f"{cores} host core(s)"
    return {"value": kept / dt if dt > 0 else None, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle Schwarz + screened J/K over a random {k} of {mol.nshell} shells "
                      f"({kept} kept quartets in {dt:.2f} s, {how})"}


def run_batch(args):
    """The batched form: every molecule's J, K, E and gradient in one call
    (one persistent kernel per class pair and band over all molecules,
    replayed as a CUDA graph), against a loop of single-molecule calls of the
    same kernels."""
    import torch
    from paper_2406_11185_gb300 import adft, parallel, synth
    ws, rank, local = _dist()
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    mols_all = synth.batch_molecules(256)
    mine = parallel.shard_molecules(len(mols_all), rank, ws)
    mols = [mols_all[i] for i in mine]
    Ds = [synth.make_density(m, synth.default_nocc(m, None), 9000 + i) for i, m in zip(mine, mols)]
    thresh, split = 1e-10, 1e-5
    t0 = time.time()
    bases = [adft.Basis.from_molecule(m) for m in mols]
    bt = adft.Batch(bases)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    Dt = [torch.from_numpy(D).to(dev) for D in Ds]
    Dp = bt.pack(Dt)
    s = torch.cuda.Stream(device=dev)
    grad = bool(args.grad)
    with torch.cuda.stream(s):
        # the launch shapes are tuned on the first 32 molecules (the same recipe)
        # and installed in the full batch
        t0 = time.time()
        nsub = min(32, len(bases))
        sub = adft.Batch(bases[:nsub])
        tab = adft.adft_batch_autotune(sub, sub.pack(Dt[:nsub]), thresh=thresh, split=split, precision="mixed",
                                       stream=s)
        adft.adft_batch_set_tuning(bt, tab)
        del sub
        tune_s = time.time() - t0
        out = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", grad=grad, stream=s)
        for _ in range(args.warmup):
            out = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", grad=grad, stream=s,
                                     out=out)
        s.synchronize()
        times = []
        with ClockSampler(dev.index or 0) as clk:
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                out = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", grad=grad,
                                         stream=s, out=out)
                b.record(s)
                b.synchronize()
                times.append(a.elapsed_time(b))
        st = adft.adft_batch_last_stats(bt)
        loop_ms = None
        if args.compare_loop:
            # the same work as a loop of single-molecule calls (default launch shapes)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for bs, D in zip(bases, Dt):
                adft.adft_jk_energy(bs, D, thresh=thresh, split=split, precision="mixed", check=False, stream=s,
                                    on_device=True)
                if grad:
                    adft.adft_jk_grad(bs, D, thresh=thresh, split=split, precision="mixed", check=False, stream=s)
            b.record(s)
            b.synchronize()
            loop_ms = a.elapsed_time(b)
    quartets = st["quartets_fp64"] + st["quartets_fp32"]
    ms_total, all_q = parallel.aggregate(float(sum(times)), quartets * args.steps, device=dev)
    ms = ms_total / args.steps
    line = {"metric": METRIC, "value": all_q / (ms_total / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batch256: {WORKLOADS['batch256']}", "molecules_per_rank": len(mols),
                       "nbf_total": int(sum(b.nbf for b in bases)), "precision": "mixed",
                       "parallelism": f"molecules sharded x{ws}", "launch_shapes": "autotuned per class pair"},
            "step": ("J, K, E and gradient" if grad else "J, K and E") + " of every molecule, one graph replay",
            "batched_s": ms / 1e3, "loop_of_single_calls_s": None if loop_ms is None else loop_ms / 1e3,
            "speedup_vs_loop": None if loop_ms is None else loop_ms / ms, "setup_s": setup_s, "autotune_s": tune_s,
            "quartets": {"fp64_band": st["quartets_fp64"], "fp32_band": st["quartets_fp32"]},
            "clocks": clk.summary(),
            # per step: D transform, screen, scan, J/K kernels per class pair and band,
            # output transform, energy, gradient kernels per class pair and band
            "gpu_launches": (5 + (4 if grad else 2) * batch_class_pairs(mols)) * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_scf(args):
    """The SCF driver around the J/K build on the workload (see --scf)."""
    import torch
    from paper_2406_11185_gb300 import adft, scf, synth
    mol, opt = synth.config(args.workload)
    split = opt["split"] if args.split is None else args.split
    out = {"workload": f"{args.workload}: {WORKLOADS.get(args.workload, '')}", "nbf": mol.nbf(),
           "nocc": int(round(float(np.sum(synth.nuclear_charges(mol))))) // 2, "thresh": opt["thresh"], "runs": []}
    for prec, inc in (("fp64", False), ("fp64", True), ("mixed", True)):
        t0 = time.time()
        rhf = scf.RHF(mol, thresh=opt["thresh"], precision=prec, split=split, incremental=inc)
        r = rhf.run(e_tol=1e-9, g_tol=1e-6)
        torch.cuda.synchronize()
        # the single-point force of the converged density (one-electron, J/K
        # and nuclear-repulsion gradients)
        tf = time.time()
        g = scf.scf_gradient(rhf, r)
        torch.cuda.synchronize()
        force_s = time.time() - tf
        full = [ms for k, ms in r["builds"] if k == "full"]
        inc_ms = [ms for k, ms in r["builds"] if k == "incremental"]
        out["runs"].append({"precision": prec, "split": split if prec == "mixed" else None, "incremental": inc,
                            "energy": r["energy"], "iterations": r["iterations"], "converged": r["converged"],
                            "wall_s": time.time() - t0, "full_builds": len(full),
                            "full_build_ms_median": float(np.median(full)) if full else None,
                            "incremental_builds": len(inc_ms),
                            "incremental_build_ms_median": float(np.median(inc_ms)) if inc_ms else None,
                            "jk_ms_total": float(sum(full) + sum(inc_ms)), "force_s": force_s,
                            "force_max_abs": float(g.abs().max().item()),
                            "net_force": float(g.sum(0).abs().max().item())})
    e64 = out["runs"][0]["energy"]
    for run in out["runs"]:
        run["energy_err_vs_full_fp64"] = abs(run["energy"] - e64)
    print(json.dumps(out), flush=True)
    return 0


def run_probe(args):
    """Untimed builds for profilers (see --probe)."""
    import torch
    from paper_2406_11185_gb300 import adft
    mol, opt, Dn = workload(args.workload)
    basis = adft.Basis.from_molecule(mol)
    D = torch.from_numpy(Dn).cuda()
    split = opt["split"] if args.split is None else args.split
    kw = {"fp64": dict(thresh=opt["thresh"], precision="fp64"),
          "fp32": dict(thresh=opt["thresh"], split=1e9, precision="mixed"),
          "mixed": dict(thresh=opt["thresh"], split=split, precision="mixed")}[args.probe]
    band = 0 if args.probe == "fp64" else 1
    tab = None
    if args.probe == "mixed":  # the benchmark's launch shapes: autotuned on the 60-atom molecule
        tname = "c60" if args.workload == "c240" else args.workload
        tmol, topt, tD = workload(tname)
        tb = adft.Basis.from_molecule(tmol) if tname != args.workload else basis
        tab = adft.adft_autotune(tb, torch.from_numpy(tD).cuda(), thresh=topt["thresh"], split=split,
                                 precision="mixed")
        adft.adft_set_tuning(basis, tab)
    if args.probe_variant is not None:
        if args.probe_cp is None:
            raise SystemExit("--probe-variant needs --probe-cp")
        if tab is None:
            tab = np.full((2, 55), 4, dtype=np.int32)
        tab[band, args.probe_cp] = tab[band, args.probe_cp] % adft.TUNE_VARIANT_STRIDE + \
            args.probe_variant * adft.TUNE_VARIANT_STRIDE
        adft.adft_set_tuning(basis, tab)
    mask = None
    if args.probe_cp is not None:
        mask = np.zeros((2, 55), np.uint8)
        mask[band, args.probe_cp] = 1
    for _ in range(args.probe_reps):
        adft.adft_jk_build(basis, D, check=False, pair_mask=mask, **kw)
    torch.cuda.synchronize()
    cs = adft.adft_jk_last_class_stats(basis)
    rows = [{"band": bd, "cp": cp, "quartets": int(cs["quartets"][bd][cp]),
             "prim_quartets": int(cs["prim_quartets"][bd][cp]), "bra_prims": int(cs["bra_prims"][bd][cp]),
             "flops_model": float(cs["flops"][bd][cp]),
             "tuning": None if tab is None else int(tab[bd][cp])}
            for bd in (0, 1) for cp in range(55) if cs["prim_quartets"][bd][cp] > 0]
    print(json.dumps({"probe": args.probe, "workload": args.workload, "class_pair": args.probe_cp,
                      "variant": args.probe_variant, "phases_ms": adft.adft_jk_last_timings(basis),
                      "classes": rows}), flush=True)
    return 0


def batch_class_pairs(mols):
    ls = sorted({l for m in mols for _, l, _, _ in m.shells})
    ncls = sum(1 for a in ls for b in ls if a >= b)
    return ncls * (ncls + 1) // 2


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    mol, opt, D = workload(args.workload)
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(mol, opt, D, budget_s=args.ref_budget)
        if i >= args.warmup:
            vals.append(r)
    v = float(np.median([r["value"] for r in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}"},
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def one_phase(basis, D, stream, flush, kw, steps, warmup, mask=None, sampler=None):
    """Per-step device times (ms) of adft_jk_energy builds: `warmup` untimed
    builds, then `steps` timed ones, each after an L2 flush, with CUDA events
    on the launching stream.  Returns (times, phases, energy tensor)."""
    import torch
    from paper_2406_11185_gb300 import adft, parallel

    def step():
        e = adft.adft_jk_energy(basis, D, check=False, on_device=True, pair_mask=mask, **kw)
        if mask is not None:  # this rank's class pairs: the sum over ranks is the energy
            parallel.sum_partials(e)
        return e

    e = None
    for _ in range(warmup):
        e = step()
    torch.cuda.synchronize()
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    times, phases = [], []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e = step()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        phases.append(adft.adft_jk_last_timings(basis))
    torch.cuda.synchronize()
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    return times, phases, e


def stored_blocks(name):
    """The oracle's sampled J/K blocks of a workload (tests/golden/<name>_blocks.json,
    written by tests/golden/make_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_blocks.json")
    return json.load(open(path)) if os.path.exists(path) else None


def blocks_error(mol, J, K, ref):
    """max |dJ|, |dK| over the stored oracle blocks."""
    o, sl = 0, []
    for _, l, _, _ in mol.shells:
        n = 2 * l + 1 if mol.spherical else (l + 1) * (l + 2) // 2
        sl.append(slice(o, o + n))
        o += n
    Jc, Kc = J.cpu().numpy(), K.cpu().numpy()
    ej = max(float(np.max(np.abs(Jc[sl[a], sl[b]] - np.array(Jb)))) for (a, b), Jb in zip(ref["pairs"], ref["J"]))
    ek = max(float(np.max(np.abs(Kc[sl[a], sl[b]] - np.array(Kb)))) for (a, b), Kb in zip(ref["pairs"], ref["K"]))
    return {"max_abs_dJ": ej, "max_abs_dK": ek, "blocks": len(ref["pairs"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=os.environ.get("ADFT_BENCH_WORKLOAD", "c240"), choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="adft", choices=["adft", "reference"])
    ap.add_argument("--ref-budget", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--split", type=float, default=None, help="FP64 band iff Q_ab Q_cd >= split (default: the "
                    "workload's)")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed builds of the plain FP64 arm (default: --steps on the 60-atom molecule, 1 on "
                         "the 2,064-function one, whose FP64 build takes minutes)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 60-atom mixed and FP64 arms reported beside a larger workload")
    ap.add_argument("--compare-loop", action="store_true",
                    help="batch256: also time the same work as a loop of single-molecule calls")
    ap.add_argument("--grad", action="store_true",
                    help="single molecule: also time one nuclear gradient (adft_jk_grad) outside the timed "
                         "steps; batch256: include the gradient of every molecule in each step")
    ap.add_argument("--probe", choices=["fp64", "fp32", "mixed"], default=None,
                    help="profiling target: untimed builds of the workload with every kept quartet in FP64 (fp64) "
                         "or in FP32 (fp32, mixed with split 1e9), default launch shapes; or the benchmark's "
                         "mixed build (mixed: the workload's split, launch shapes autotuned as in the benchmark); "
                         "then per-class statistics as JSON (the command the ncu summaries under profiles/ run)")
    ap.add_argument("--probe-variant", type=int, default=None, help="with --probe-cp: run that class pair with "
                    "this kernel variant (adft_set_tuning)")
    ap.add_argument("--probe-cp", type=int, default=None, help="with --probe: evaluate only this class pair "
                    "X(X+1)/2 + Y (a pair mask), for single-kernel captures")
    ap.add_argument("--probe-reps", type=int, default=2, help="with --probe: number of builds")
    ap.add_argument("--scf", action="store_true",
                    help="run the closed-shell SCF driver (scf.RHF) on the workload and print its iterations, "
                         "energy, J/K build times (full and incremental) and the single-point force as one JSON "
                         "line")
    args = ap.parse_args()
    if args.scf:
        return run_scf(args)
    if args.probe:
        return run_probe(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        return run_batch(args)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2406_11185_gb300 import adft, parallel

    t0 = time.time()
    mol, opt, Dn = workload(args.workload)
    basis = adft.Basis.from_molecule(mol)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    D = torch.from_numpy(Dn).to(dev)
    thresh = opt["thresh"]
    split = opt["split"] if args.split is None else args.split
    prec = args.precision
    kw = dict(thresh=thresh, split=split, precision=prec)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    # measured ALU peaks of this GPU (the roofline denominators)
    peaks = {"fp64": adft.adft_alu_peak(True, 4000), "fp32": adft.adft_alu_peak(False, 20000)}

    # launch shapes: autotuned on the 60-atom molecule of the same recipe (its
    # kernels cover the same class pairs in seconds) and installed here
    t0 = time.time()
    tune_name = "c60" if args.workload == "c240" else args.workload
    if tune_name != args.workload:
        tmol, topt, tD = workload(tune_name)
        tbasis = adft.Basis.from_molecule(tmol)
        tDt = torch.from_numpy(tD).to(dev)
    else:
        tmol, topt, tbasis, tDt = mol, opt, basis, D
    tab64, ms64 = adft.adft_autotune(tbasis, tDt, thresh=topt["thresh"], precision="fp64", return_times=True)
    tab, tune_ms = adft.adft_autotune(tbasis, tDt, thresh=topt["thresh"], split=split, precision=prec,
                                      return_times=True)
    adft.adft_set_tuning(basis, tab)
    tune_s = time.time() - t0
    mask = parallel.class_pair_masks(tune_ms, ws, rank, device=dev) if ws > 1 else None

    # ---- the timed arm (the metric): K steps after W warm-up steps
    with ClockSampler(dev.index or 0) as clk:
        times, phases, e = one_phase(basis, D, stream, flush, kw, args.steps, args.warmup, mask)
    Emain = float(e.item())
    st = adft.adft_jk_last_stats(basis)
    cls = adft.adft_jk_last_class_stats(basis)
    quartets = st["quartets_fp64"] + st["quartets_fp32"]
    _, prim_all = parallel.aggregate(0.0, float(st["prim_quartets_fp64"] + st["prim_quartets_fp32"]), device=dev)
    cart_eris = float(np.sum(cls["quartets"] * cartesian_block_sizes()[None, :]))
    ms_total, all_quartets = parallel.aggregate(float(sum(times)), quartets * args.steps / ws, device=dev)
    ms = ms_total / args.steps
    value = all_quartets / (ms_total / 1e3)
    ph = {k: float(np.mean([p[k] for p in phases])) for k in phases[0]}

    # ---- accuracy of this build: stored oracle blocks (sampled J and K)
    ref_blocks = stored_blocks(args.workload)
    J, K = adft.adft_jk_build(basis, D, check=False, **kw)
    acc = {"vs_oracle_blocks": blocks_error(mol, J, K, ref_blocks) if ref_blocks and mask is None else None}
    del J, K

    # ---- end to end through the C ABI with host buffers: pinned D in, J and K out
    Dh = torch.from_numpy(Dn).pin_memory()
    Jh = torch.empty_like(Dh).pin_memory()
    Kh = torch.empty_like(Dh).pin_memory()
    Jd, Kd, Dd = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
    e2e_ms = []
    # the first pass warms the copies and pinned buffers (the kernels are warm); where one build
    # takes a minute that warm-up is negligible and both passes are timed
    first_timed = 0 if args.workload == "c240" else 1
    for i in range(first_timed + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Dd.copy_(Dh, non_blocking=True)
        adft.adft_jk_build(basis, Dd, check=False, out=(Jd, Kd), pair_mask=mask, **kw)
        if mask is not None:
            parallel.sum_partials(Jd, Kd)  # the exchange step: J and K summed over ranks
        Jh.copy_(Jd, non_blocking=True)
        Kh.copy_(Kd, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= first_timed:
            e2e_ms.append(a.elapsed_time(b))
    nb2 = Dn.size * 8
    e2e_ms_max, _ = parallel.aggregate(float(np.median(e2e_ms)), 0.0, device=dev)

    # ---- the plain FP64 arm of the same molecule (mixed vs FP64 at the energy budget)
    fp64_arm = None
    if prec == "mixed":
        n64 = args.fp64_steps if args.fp64_steps is not None else (1 if args.workload == "c240" else args.steps)
        w64 = 0 if args.workload == "c240" else args.warmup  # FP64 kernels were warmed by the autotuner
        if n64 > 0:
            adft.adft_set_tuning(basis, tab64)
            t64, ph64, e64 = one_phase(basis, D, stream, flush, dict(thresh=thresh, precision="fp64"), n64, w64,
                                       mask)
            E64 = float(e64.item())
            fp64_arm = {"workload": args.workload, "steps": n64, "warmup": w64,
                        "median_s": float(np.median(t64)) / 1e3, "min_s": float(np.min(t64)) / 1e3,
                        "energy": E64, "energy_err_mixed_vs_fp64": abs(Emain - E64)}
            if ref_blocks and mask is None:
                J, K = adft.adft_jk_build(basis, D, check=False, thresh=thresh, precision="fp64")
                fp64_arm["vs_oracle_blocks"] = blocks_error(mol, J, K, ref_blocks)
                del J, K
            adft.adft_set_tuning(basis, tab)

    # ---- roofline of the dominant kernel group (the ALU-bound ERI kernels of a band)
    # traffic: DRAM bytes (read + write) of the band's class-pair launches in one
    # build, from one ncu capture of the current kernels; null until the kernels
    # changed by the long-range operator option are captured again (the capture
    # of the version before it: 1.74 GB FP32 band, 61.0 GB FP64 band per c240
    # build at split 3e-3)
    traffic = {}
    groups = {"eri_fp32": (ph["eri_fp32_ms"], float(cls["flops"][1].sum()), peaks["fp32"]["tflops"], "FP32"),
              "eri_fp64": (ph["eri_fp64_ms"], float(cls["flops"][0].sum()), peaks["fp64"]["tflops"], "FP64")}
    dom = max(groups, key=lambda k: groups[k][0])
    gms, gfl, gpk, gkind = groups[dom]
    ach = gfl / (gms / 1e3) / 1e12 if gms > 0 else 0.0
    roof = {"bound": "alu", "kernel": f"{dom} (all class-pair launches of the band)", "achieved": ach,
            "peak": gpk, "unit": "TFLOP/s", "frac": ach / gpk if gpk else None, "traffic": traffic.get(dom),
            "traffic_unit": "bytes per build (all launches of the band)",
            "peak_kind": f"measured in this run: adft_alu_peak ({gkind} FMA chains on every SM)",
            "flops_model": "class_flops per evaluated primitive quartet, bra primitive and quartet",
            "other": {k: {"ms": v[0], "tflops": (v[1] / (v[0] / 1e3) / 1e12) if v[0] > 0 else 0.0,
                          "peak": v[2], "frac": ((v[1] / (v[0] / 1e3) / 1e12) / v[2]) if v[0] > 0 and v[2] else 0.0}
                      for k, v in groups.items()}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32+f64" if prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "nbf": basis.nbf,
                       "natom": mol.natom, "nshell": mol.nshell, "thresh": thresh, "split": split,
                       "precision": prec, "l2": "flushed before every step (256 MB write)",
                       "parallelism": ("single GPU" if ws == 1 else
                                       f"class pairs sharded x{ws} (longest processing time on the measured "
                                       "kernel times), one sum all-reduce of E per step (of J and K end to end)"),
                       "launch_shapes": f"autotuned per class pair on {tune_name}"},
            "jk_build_s": ms / 1e3, "jk_build_s_fp64": None if fp64_arm is None else fp64_arm["median_s"],
            "speedup_vs_fp64": None if fp64_arm is None else fp64_arm["median_s"] * 1e3 / ms,
            "energy": Emain, "energy_fp64": None if fp64_arm is None else fp64_arm["energy"],
            "energy_err_vs_fp64": None if fp64_arm is None else fp64_arm["energy_err_mixed_vs_fp64"],
            "fp64_arm": fp64_arm, "accuracy": acc, "autotune_s": tune_s,
            "quartets": {"fp64_band": st["quartets_fp64"], "fp32_band": st["quartets_fp32"],
                         "unique_before_screening": st["quartets_total"],
                         "prim_fp64_band": st["prim_quartets_fp64"], "prim_fp32_band": st["prim_quartets_fp32"]},
            "throughput": {"screened_quartets_per_s": value, "cartesian_eris_per_s": cart_eris / (ms / 1e3),
                           "primitive_quartets_per_s": prim_all / (ms / 1e3)},
            "step_ms": {"mean": ms, "median": float(np.median(times)), "min": float(np.min(times)),
                        "max": float(np.max(times))},
            "phases_ms": ph, "setup_s": setup_s, "peaks": peaks,
            "clocks": clk.summary(),
            "e2e": {"value": quartets / (e2e_ms_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": nb2,
                    "d2h_bytes_per_step": 2 * nb2, "ms": e2e_ms_max, "samples": len(e2e_ms)},
            "gpu_launches": (launches_per_step(basis_classes(mol), mixed=prec == "mixed") if mask is None else
                             5 + int(np.count_nonzero(mask))) * args.steps,
            "roofline": roof}

    # ---- the 60-atom molecule beside a larger workload: mixed and FP64 arms
    # with the same steps and warm-up (both medians)
    if args.workload != "c60" and not args.no_secondary and mask is None and prec == "mixed":
        smol, sopt, sDn = workload("c60")
        sb = tbasis if tune_name == "c60" else adft.Basis.from_molecule(smol)
        sD = torch.from_numpy(sDn).to(dev)
        skw = dict(thresh=sopt["thresh"], split=split, precision="mixed")
        adft.adft_set_tuning(sb, tab)
        tm, _, em = one_phase(sb, sD, stream, flush, skw, args.steps, args.warmup)
        adft.adft_set_tuning(sb, tab64)
        t64, _, e64 = one_phase(sb, sD, stream, flush, dict(thresh=sopt["thresh"], precision="fp64"), args.steps,
                                args.warmup)
        ssts = adft.adft_jk_last_stats(sb)
        q = ssts["quartets_fp64"] + ssts["quartets_fp32"]
        Jm, Km = adft.adft_jk_build(sb, sD, check=False, **skw)
        sref = stored_blocks("c60")
        line["c60"] = {"workload": f"c60: {WORKLOADS['c60']}", "split": split, "steps": args.steps,
                       "warmup": args.warmup, "mixed_median_s": float(np.median(tm)) / 1e3,
                       "fp64_median_s": float(np.median(t64)) / 1e3,
                       "speedup_vs_fp64": float(np.median(t64)) / float(np.median(tm)),
                       "screened_quartets_per_s": q / (float(np.median(tm)) / 1e3),
                       "energy_err_mixed_vs_fp64": abs(float(em.item()) - float(e64.item())),
                       "mixed_vs_oracle_blocks": blocks_error(smol, Jm, Km, sref) if sref else None}
    if args.grad:
        # one gradient of E_JK at the same D and options (outside the timed steps)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g = adft.adft_jk_grad(basis, D, check=False, pair_mask=mask, **kw)
        if mask is not None:
            parallel.sum_partials(g)
        b.record(stream)
        b.synchronize()
        line["gradient"] = {"s": a.elapsed_time(b) / 1e3, "precision": prec,
                            "max_abs": float(g.abs().max().item()),
                            "net_force": float(g.sum(0).abs().max().item()),
                            "phases_ms": adft.adft_jk_last_timings(basis)}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(mol, opt, Dn)
        one = cpu_oracle_rate(mol, opt, Dn, budget_s=8.0, nthreads=1, growth=1.25)
        line["cpu_baseline"]["single_core"] = {k: one[k] for k in ("value", "cores", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def basis_classes(mol):
    """Number of non-empty pair classes (l_a >= l_b) of the molecule."""
    ls = sorted({l for _, l, _, _ in mol.shells})
    present = set()
    for a in ls:
        for b in ls:
            if a >= b:
                present.add((a, b))
    return len(present)


def cartesian_block_sizes():
    """Cartesian integrals per shell quartet of every class pair X(X+1)/2 + Y,
    class X = l_a(l_a+1)/2 + l_b (l_a >= l_b, l <= 3): [55]."""
    nc = [(l + 1) * (l + 2) // 2 for l in range(4)]
    cls = [nc[la] * nc[lb] for la in range(4) for lb in range(la + 1)]
    return np.array([cls[x] * cls[y] for x in range(len(cls)) for y in range(x + 1)], dtype=np.float64)


def launches_per_step(ncls, mixed=True):
    """Kernels of one adft_jk_energy call: D transform, screen, scan, one ERI
    kernel per class pair and band, output transform, energy."""
    ncp = ncls * (ncls + 1) // 2
    return 5 + ncp * (2 if mixed else 1)


if __name__ == "__main__":
    sys.exit(main())
