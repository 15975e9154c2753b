#!/usr/bin/env python
"""Benchmark of the block-sparse MPS eigensolver hot path on GB300.

Default workload (the JSON contract): the open Hubbard chain L = 32 (64
spin-orbital sites), half filling, t = 1, U = 4, maximal rank r_max = 256,
from a random iterate of full rank 256 (seed 1).  One step = one pass of Alg. 2
(exact Rayleigh quotient, zip-up MPO applies of the preconditioned terms,
error-controlled residual sum with rank truncations, 2x2 Rayleigh-Ritz,
truncation of the update).  W untimed warm-up steps, then K timed steps, each
profiled per kernel kind with CUDA events on the library's stream.

value: MPO.MPS apply throughput, TFLOP/s: the algorithmic flops of the zip-up
contraction stage (sum of 2mnk over its grouped-GEMM work list, which includes
the MPO channel combine) over that stage's device time in the timed steps.
The whole step's algorithmic flops and time are reported beside it ("step").
--precision tf32x3 runs the contraction on the tensor cores in split precision
(the solver's policy falls back to FP64 once the split error estimate nears the
residual tolerance).

Other workloads (--workload):
  tta_learned   time to |E - E_ref| <= 1e-8 Eh on the config-1 chain from e_1,
                FP64 / split precision x plain / learned controller parameters
  tta_k12       the same chain from its random rank-32 start, golden constants
  hubbard_tta   the config-2 trajectory from e_1 (time to rho <= 1e-8 or to the
                settled energy)
  hubbard_e1    Alg. 2 steps of that trajectory
  batched       128 independent Hamiltonians: recorded CUDA graph, one batched
                call, one call per instance
  mlp           the controller network's training step on the tensor cores
  coulomb14_alg3, coulomb14_alg4_D4   the paper's K = 14 Coulomb-like runs
  ozaki_gemm    the FP64 GEMM emulated on the tensor cores vs cuBLAS DGEMM
  profile_step, profile_apply, profile_truncation   fixed runs for profilers
--jacobi-precond sets the k from which truncation SVDs start from an FP32
Jacobi (0: never).
Usage (contract): python bench.py --gpus N --steps K --warmup W [--impl reference]
"""

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # the oracle baseline runs on one host core

import argparse
import json
import math
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPO·MPS apply TFLOP/s (% roofline); time to 1e-8 Eh, mixed+learned vs FP64"
WORKLOAD = ("hubbard_chain L=32 (K=64 spin-orbital sites), n_up=n_dn=16, t=1, U=4, r_max=256, "
            "Alg. 2 steps from a random iterate of full rank 256 (seed 1)")
WORKLOAD_E1 = ("hubbard_chain L=32 (K=64 spin-orbital sites), n_up=n_dn=16, t=1, U=4, r_max=256, FP64, "
               "Alg. 2 trajectory from e_1")
L2_FLUSH_BYTES = 256 << 20


def load_params(L=32):
    path = os.path.join(ROOT, "tests", "golden", f"bench_params_hubbard_L{L}.json")
    with open(path) as f:
        return json.load(f)


def setup(ctx, nat, seed, L=32, r_max=256):
    from paper_2604_16118_gb300 import problem
    from synth import hubbard_chain, random_block_values
    prm = load_params(L)
    wl = hubbard_chain(L=L, r_max=r_max)
    n = L // 2
    gamma = problem.hubbard_shift(wl.h, n, n, margin=1.0)
    th = problem.theta_diagonal(wl.h, wl.eri, 1, L, gamma)
    tmin, tmax = problem.spectrum_bounds(th, 1, n, n)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 1, 2 * n, gamma)
    p = nat.make_precond(th, tmin, tmax, prm["c0"], prm["alpha0"])
    sp = nat.solver_params(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"], tau=1e-8,
                           r_max=r_max)
    if seed is None:
        x = nat.mps_create(ctx, L, 1, n, n)                    # e_1
    else:
        nval = nat.mps_random_size(L, 1, n, n, r_max)
        x = nat.mps_create(ctx, L, 1, n, n, r_max, random_block_values(nval, seed))
    return dict(wl=wl, W=W, p=p, sp=sp, x=x, gamma=gamma, theta=th, tmin=tmin, tmax=tmax, prm=prm)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp64_gemm_peak(torch, dev):
    """cuBLAS FP64 GEMM throughput (TFLOP/s), best of 5 (4096^3)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    return best


def oracle_steps(n_steps, L=32, r_max=256):
    """The oracle (as it stands) on the same trajectory: per-step wall times."""
    from oracle import bsmps as OB
    from oracle import fermion as OF
    from oracle import mpo as OM
    from oracle import pinvit as OPI
    from oracle import precond as OP
    from synth import hubbard_chain
    prm = load_params(L)
    wl = hubbard_chain(L=L, r_max=r_max)
    n = L // 2
    gamma = 1.0 - OP.energy_lower_bound(wl.h, wl.eri, 1, n, n, cholesky=False)
    W = OM.build_mpo(wl.h, wl.eri, 1, 2 * n, gamma)
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, 1)
    species = OF.site_species(L, 1)
    th = OP.theta_diag(t_so, v_so, 2 * n, gamma, 2 * L)
    tmin, tmax = OP.spectrum_bounds(th, species, (n, n))
    prec = OP.Preconditioner(th, tmin, tmax, prm["c0"], prm["alpha0"])
    params = OPI.SolverParams(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"], tau=1e-8,
                              r_max=r_max)
    st = OPI.SolverState()
    x = OB.e1_mps(species, (n, n))
    times, energies = [], []
    for _ in range(n_steps):
        t0 = time.perf_counter()
        x, info = OPI.step(x, W, prec, params, st)
        times.append(time.perf_counter() - t0)
        energies.append(info["lambda"] - gamma)
    return times, energies


def gpu_step_flops(nat, ctx, n_steps):
    """Algorithmic flops of steps 0..n_steps-1 from e_1, counted by the library."""
    S = setup(ctx, nat, seed=None)
    st = nat.solver_state()
    x = S["x"]
    out = []
    for _ in range(n_steps):
        x, info = nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], st, x)
        out.append(info["flops"])
    return out


ORACLE_APPLY_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import bsmps as OB, fermion as OF, mpo as OM, precond as OP
from synth import hubbard_chain, random_block_values
L, r, seed, shift, reps = {L}, {r}, {seed}, {shift}, {reps}
wl = hubbard_chain(L=L, r_max=r)
n = L // 2
gamma = 1.0 - OP.energy_lower_bound(wl.h, wl.eri, 1, n, n, cholesky=False)
W = OM.build_mpo(wl.h, wl.eri, 1, 2 * n, gamma)
species = OF.site_species(L, 1)
dims = OB.default_dims(species, (n, n), r)
size = OB.BSMPS(species, (n, n), dims, [dict() for _ in species]).layout()[1]
x = OB.BSMPS.from_flat(species, (n, n), dims, random_block_values(size, seed))
times = []
for _ in range(reps):
    t0 = time.perf_counter()
    OB.apply_zipup(W, x, shift=shift)
    times.append(time.perf_counter() - t0)
print(json.dumps(times))
"""


def oracle_apply_times(cores, reps=1, L=32, r=256, seed=1, shift=-70.0):
    """The oracle's zip-up application of one preconditioner branch of the full-rank
    iterate, timed in a fresh interpreter whose BLAS uses `cores` threads."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    code = ORACLE_APPLY_SNIPPET.format(root=ROOT, L=L, r=r, seed=seed, shift=shift, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def apply_flops_per_branch(nat, ctx, S):
    """Algorithmic flops of the zip-up contraction for one branch of the iterate
    S["x"] (counted by the library from its work list)."""
    ctx.profile(True)
    nat.apply_zipup(ctx, S["W"], S["x"], shift=-70.0)
    st = ctx.kernel_stats(reset=True)
    ctx.profile(False)
    return st["apply"][2]


def run_reference(args):
    """The oracle arm: each step is the oracle's zip-up application of one
    preconditioner branch of the full-rank iterate (a bounded sample of the
    default workload's apply, timed on the host cores); value in the same unit
    as the GPU arm's (apply TFLOP/s), flops counted by the library."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.warmup + args.steps
    cores = os.cpu_count() or 1
    times = oracle_apply_times(1, reps=n)
    tm = times[args.warmup:]
    fl = None
    note = None
    try:
        from paper_2604_16118_gb300 import build, native as nat
        build.build()
        ctx = nat.Context(0)
        fl = apply_flops_per_branch(nat, ctx, setup(ctx, nat, seed=1))
    except Exception as e:
        note = "flop count needs the library on a GPU: " + str(e).splitlines()[0]
    val = fl * len(tm) / sum(tm) / 1e12 if fl else None
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(tm)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "oracle zip-up apply of one preconditioner branch",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1, "host_cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed zip-up applications (after {args.warmup} untimed) "
                                       "of one branch of the rank-256 iterate, numpy FP64 oracle, BLAS on 1 thread"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if note:
        line["note"] = note
    print(json.dumps(line))
    return 0


JOINT_WORKLOAD = ("coulomb_1d K=14 N=4 gamma=4 (the simultaneous-eigenvalue experiment of Sec. 7.2), D=4, "
                  "Alg. 4 on a joint block MPS from the 4 lowest determinants, FP64")


def setup_joint(ctx, nat):
    from paper_2604_16118_gb300 import problem
    from synth import coulomb_1d
    with open(os.path.join(ROOT, "tests", "golden", "bench_params_coulomb14_D4.json")) as f:
        prm = json.load(f)
    K, N, gamma, D = 14, 4, 4.0, 4
    wl = coulomb_1d(K=K, N=N, n_grid=8192)
    th = problem.theta_diagonal(wl.h, wl.eri, 0, N, gamma)
    tmin, tmax = problem.spectrum_bounds(th, 0, N, 0, h=wl.h)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, N, gamma)
    p = nat.make_precond(th, tmin, tmax, prm["c0"], prm["alpha0"])
    sp = nat.solver_params(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"], tau=1e-10)
    occ = problem.lowest_determinants(np.diag(wl.h), 0, N, 0, D)
    x = nat.mps_create_joint(ctx, K, 0, N, 0, D, occ=occ)
    return dict(wl=wl, W=W, p=p, sp=sp, x=x, gamma=gamma, prm=prm, K=K, N=N, D=D, occ=occ)


def oracle_joint_step0():
    """The oracle's first Alg. 4 step of the joint workload (wall seconds, Ritz values)."""
    from oracle import fermion as OF
    from oracle import joint as OJ
    from oracle import mpo as OM
    from oracle import pinvit as OPI
    from oracle import precond as OP
    from synth import coulomb_1d
    with open(os.path.join(ROOT, "tests", "golden", "bench_params_coulomb14_D4.json")) as f:
        prm = json.load(f)
    K, N, gamma, D = 14, 4, 4.0, 4
    wl = coulomb_1d(K=K, N=N, n_grid=8192)
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = OP.theta_diag(t_so, v_so, N, gamma, K)
    species = OF.site_species(K, 0)
    tmin, tmax = OP.spectrum_bounds(th, species, (N, 0), t_diag=np.diag(wl.h))
    prec = OP.Preconditioner(th, tmin, tmax, prm["c0"], prm["alpha0"])
    W = OM.build_mpo(wl.h, wl.eri, 0, N, gamma)
    params = OPI.SolverParams(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"], tau=1e-10)
    x = OJ.from_determinants(species, (N, 0), OJ.lowest_determinants(species, (N, 0), np.diag(wl.h), D))
    t0 = time.perf_counter()
    x, info = OJ.step(x, W, prec, params, OPI.SolverState())
    return time.perf_counter() - t0, info["lambda"]


def main_joint(args):
    """Alg. 4 steps of the joint workload: W untimed, K timed (device events,
    L2 flushed between steps); step 0 is timed separately against the oracle."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    S = setup_joint(ctx, nat)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = nat.solver_state()
    x = S["x"]

    def timed(xx):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xx, info = nat.eigensolve_joint_step(ctx, S["W"], S["p"], S["sp"], st, xx)
        e1.record(stream)
        e1.synchronize()
        return xx, info, e0.elapsed_time(e1)

    x, info0, ms0 = timed(x)                      # step 0 (compared with the oracle below)
    for _ in range(max(args.warmup - 1, 0)):
        x, _ = nat.eigensolve_joint_step(ctx, S["W"], S["p"], S["sp"], st, x)
    ctx.sync()
    x_after_warmup = (x.export(), x.bonds(), st.eta_res, st.n)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    total_ms, total_flops, infos = 0.0, 0.0, []
    for _ in range(args.steps):
        x, info, ms = timed(x)
        total_ms += ms
        total_flops += info["flops"]
        infos.append(info)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    clocks = sampler.stop()
    ctx.profile(True)
    x, _ = nat.eigensolve_joint_step(ctx, S["W"], S["p"], S["sp"], st, x)
    stats = ctx.kernel_stats(reset=True)
    ctx.profile(False)
    name, (nl, kms, kfl, kby) = max(stats.items(), key=lambda kv: kv[1][1])
    # end to end through the C ABI with host buffers, from the post-warm-up iterate
    hx, bonds, st.eta_res, st.n = x_after_warmup
    pinned = torch.empty(len(hx), dtype=torch.float64).pin_memory()
    pinned.numpy()[:] = hx
    h2d = d2h = 0
    e2e_flops = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd = nat.mps_import(ctx, S["K"], 0, S["N"], 0, bonds, pinned.numpy())
        h2d += 8 * len(pinned)
        xd, info = nat.eigensolve_joint_step(ctx, S["W"], S["p"], S["sp"], st, xd)
        e2e_flops += info["flops"]
        out = xd.export()
        d2h += 8 * len(out)
        bonds = xd.bonds()
        pinned = torch.from_numpy(out).pin_memory()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    fp64 = fp64_gemm_peak(torch, dev)
    lam_exact = S["prm"]["lambda_exact"][:S["D"]]
    last = infos[-1] if infos else info0
    out = {
        "metric": "Alg. 4 step, algorithmic FP64 TFLOP/s", "value": total_flops / (total_ms * 1e-3) / 1e12,
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": JOINT_WORKLOAD, "step": "one Alg. 4 step",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single"},
        "gpu_launches": launches, "clocks": clocks,
        "e2e": {"value": e2e_flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d // max(args.steps, 1),
                "d2h_bytes_per_step": d2h // max(args.steps, 1), "steps": args.steps},
        "roofline": {"bound": "alu", "kernel": name, "achieved": (kfl / (kms * 1e-3) / 1e12) if kms else None,
                     "peak": fp64, "unit": "TFLOP/s", "frac": (kfl / (kms * 1e-3) / 1e12 / fp64) if kms else None,
                     "traffic": None, "peak_source": "cuBLAS FP64 GEMM 4096^3 measured in this run",
                     "launches": nl, "kernel_ms": kms},
        "kernels": {k: {"launches": v[0], "ms": v[1], "flops": v[2], "bytes": v[3]} for k, v in stats.items()},
        "steps_info": [{"lambda": [float(v) for v in i["lambda"]], "rho1": float(i["rho"][0]),
                        "eta_tries": i["eta_tries"], "max_rank": i["max_rank"], "flops": i["flops"]}
                       for i in [info0] + infos],
        "lambda_exact": lam_exact,
        "step0_ms": ms0,
    }
    if rank == 0 and not args.no_cpu_baseline:
        t_or, lam_or = oracle_joint_step0()
        out["cpu_baseline"] = {"value": info0["flops"] / t_or / 1e12, "unit": "TFLOP/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"step 0 of the same trajectory ({t_or:.1f} s; numpy FP64 oracle, "
                                         f"BLAS on 1 thread); the GPU's step 0 took {ms0:.1f} ms",
                               "lambda_match": float(np.max(np.abs(np.asarray(lam_or) - info0["lambda"])))}
    print(json.dumps(out))
    return 0


def main_ozaki(args):
    """FP64 GEMM emulated on the bf16 tensor cores (Ozaki scheme, 8 slices) vs
    cuBLAS DGEMM on the same operands; square sizes, inputs resident, events on
    the library stream, L2 flushed between repetitions."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks, src = measured_peaks()
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    rows = []
    for n in (2048, 4096):
        A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
        B = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
        C = torch.empty(n, n, dtype=torch.float64, device=dev)

        def timed(fn):
            ms = []
            for it in range(args.warmup + args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                if it >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            return float(np.median(ms))

        def emulated():
            nat.gemm_ozaki(ctx, A, B, C, 8)

        def dgemm():
            with torch.cuda.stream(stream):
                torch.matmul(A, B, out=Cd)

        Cd = torch.empty_like(C)
        ms_oz = timed(emulated)
        ms_d = timed(dgemm)
        torch.cuda.synchronize()
        scale = (A.abs() @ B.abs()).max().item()
        err = (C - Cd).abs().max().item() / scale
        fl = 2.0 * n ** 3
        pairs = 36                           # slice products of 8 slices with p + q <= 9
        rows.append({"n": n, "emulated_ms": ms_oz, "dgemm_ms": ms_d,
                     "emulated_tflops_fp64_equiv": fl / (ms_oz * 1e-3) / 1e12,
                     "dgemm_tflops": fl / (ms_d * 1e-3) / 1e12,
                     "bf16_tflops_issued": pairs * fl / (ms_oz * 1e-3) / 1e12,
                     "max_err_rel_to_abs_product": err})
        del A, B, C, Cd
    big = rows[-1]
    bf16_peak = peaks.get("bf16_tflops")
    out = {"metric": "FP64 GEMM emulated on tensor cores, FP64-equivalent TFLOP/s", "value":
           big["emulated_tflops_fp64_equiv"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": big["emulated_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 (bf16 slices, fp32 exact accumulation)", "data": "synthetic",
           "config": {"workload": "square FP64 GEMM n = 2048, 4096, standard normal entries, 8 slices",
                      "l2": "flushed between repetitions (256 MB write)"},
           "roofline": {"bound": "tensor", "kernel": "k_oz_gemm (all five launches timed together)",
                        "achieved": big["bf16_tflops_issued"], "peak": bf16_peak, "unit": "TFLOP/s",
                        "frac": big["bf16_tflops_issued"] / bf16_peak if bf16_peak else None, "traffic": None,
                        "peak_source": f"bf16 dense, {src}"},
           "sizes": rows}
    print(json.dumps(out))
    return 0


def main_outer(args):
    """Time to solution of the paper's K = 14 run: Alg. 3 (alpha = 1) from e_1 to
    the relative eigenvalue bound tau = 1e-10 (Sec. 7.2), constants as stored for
    this model (c, delta, alpha_0 by exact diagonalisation)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build, problem
    build.build()
    from paper_2604_16118_gb300 import native as nat
    from synth import coulomb_1d
    with open(os.path.join(ROOT, "tests", "golden", "bench_params_coulomb14_D4.json")) as f:
        prm = json.load(f)
    with open(os.path.join(ROOT, "tests", "golden", "paper_coulomb1d.json")) as f:
        paper = json.load(f)
    K, N, gamma = 14, 4, 4.0
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    wl = coulomb_1d(K=K, N=N, n_grid=8192)
    th = problem.theta_diagonal(wl.h, wl.eri, 0, N, gamma)
    tmin, tmax = problem.spectrum_bounds(th, 0, N, 0, h=wl.h)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, N, gamma)
    p = nat.make_precond(th, tmin, tmax, prm["c0"], prm["alpha0"])
    sp = nat.solver_params(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"])
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    fl0 = 0.0
    t0 = time.perf_counter()
    x = nat.mps_create(ctx, K, 0, N, 0)            # e_1
    y, recs, ok = nat.eigensolve_outer(ctx, W, p, sp, x, 1e-10, alpha=1.0, max_outer=40, max_inner=200)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    lam = recs[-1]["lambda"] if recs else None
    inner = sum(r["inner_steps"] for r in recs)
    fl = sum(r["flops"] for r in recs)
    out = {"metric": "time to tau = 1e-10 (Alg. 3 from e_1, relative eigenvalue bound)", "value": wall, "unit": "s",
           "n_gpus": 1, "steps": inner, "warmup": 0, "ms_per_step": 1e3 * wall / max(inner, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "coulomb_1d K=14 N=4 gamma=4 (Sec. 7.2), finite-difference orbitals, n_grid=8192",
                      "l2": "not flushed (one solve)"},
           "clocks": clocks, "converged": ok, "outer_steps": len(recs), "inner_steps": inner,
           "lambda": lam, "lambda_exact_same_discretisation": prm["lambda_exact"][0],
           "lambda_printed": paper["K14"]["lambda1_inner_outer"],
           "releig_bound": recs[-1]["releig_bound"] if recs else None,
           "max_rank": max(r["max_rank_before"] for r in recs) if recs else None,
           "tflops": fl / wall / 1e12 if wall > 0 else None,
           "e2e": {"value": wall, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main_e1(args):
    """Alg. 2 steps W..W+K-1 of the trajectory from e_1 (Sec. 7.1.4), FP64."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat

    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    S = setup(ctx, nat, seed=None)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = nat.solver_state()
    x = S["x"]

    def one_step(xx):
        return nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], st, xx)

    for _ in range(args.warmup):
        x, _ = one_step(x)
    ctx.sync()
    x_after_warmup = (x.export(), x.bonds(), st.eta_res, st.n)

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    total_ms = 0.0
    total_flops = 0.0
    infos = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = one_step(x)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_flops += info["flops"]
        infos.append(info)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    from paper_2604_16118_gb300 import replicas
    total_ms, total_flops = replicas.reduce_timing(total_ms, total_flops, dist, dev)
    clocks = sampler.stop()
    ms_per_step = total_ms / args.steps
    value = total_flops / (total_ms * 1e-3) / 1e12

    # per-kernel roofline from one profiled step (events around every launch)
    ctx.profile(True)
    x, _ = one_step(x)
    stats = ctx.kernel_stats(reset=True)
    ctx.profile(False)
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    name, (nl, kms, kfl, kby) = dom

    # end to end through the C ABI with host buffers: the same K steps again from
    # the post-warm-up iterate, uploaded from and read back to pinned host memory
    e2e_steps = args.steps
    hx, bonds, st.eta_res, st.n = x_after_warmup
    pinned = torch.empty(len(hx), dtype=torch.float64).pin_memory()
    pinned.numpy()[:] = hx
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_flops = 0.0
    for _ in range(e2e_steps):
        xd = nat.mps_import(ctx, 32, 1, 16, 16, bonds, pinned.numpy())
        h2d += 8 * len(pinned)
        xd, info = one_step(xd)
        e2e_flops += info["flops"]
        out = xd.export()
        d2h += 8 * len(out)
        bonds = xd.bonds()
        pinned = torch.from_numpy(out).pin_memory()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = e2e_flops / e2e_s / 1e12

    peaks, src = measured_peaks()
    fp64 = fp64_gemm_peak(torch, dev)
    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_E1, "step": "one Alg. 2 step", "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d // e2e_steps,
                "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps},
        "roofline": {"bound": "alu", "kernel": name, "achieved": (kfl / (kms * 1e-3) / 1e12) if kms else None,
                     "peak": fp64, "unit": "TFLOP/s", "frac": None, "traffic": None,
                     "peak_source": "cuBLAS FP64 GEMM 4096^3 measured in this run",
                     "launches": nl, "kernel_ms": kms, "kernel_bytes": kby,
                     "achieved_gbs": kby / (kms * 1e-3) / 1e9 if kms else None,
                     "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": src},
        "kernels": {k: {"launches": v[0], "ms": v[1], "flops": v[2], "bytes": v[3]} for k, v in stats.items()},
        "steps_info": [{"lambda": i["lambda"], "rho": i["rho"], "eta_tries": i["eta_tries"],
                        "max_rank": i["max_rank"], "flops": i["flops"]} for i in infos],
        "energy": infos[-1]["lambda"] - S["gamma"] if infos else None,
    }
    r = out["roofline"]
    if r["achieved"] is not None and r["peak"]:
        r["frac"] = r["achieved"] / r["peak"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = args.warmup + args.steps
        times, energies = oracle_steps(n)
        tm = times[args.warmup:]
        out["cpu_baseline"] = {"value": total_flops / sum(tm) / 1e12, "unit": "TFLOP/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"the identical Alg. 2 steps {args.warmup}..{n - 1} from e_1 "
                                         f"({sum(tm):.2f} s; numpy FP64 oracle, BLAS on 1 thread)",
                               "energy_match": abs(energies[-1] - out["energy"])}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


TF32_PER_BF16 = 1.1 / 2.25     # nominal dense TF32 / BF16 tensor rates of the chip


def kind_peak(kind, precision, fp64, peaks, src):
    """Roofline denominator of a kernel kind: the split-precision contraction
    against the TF32 tensor peak (measured BF16 peak x nominal TF32/BF16 ratio)
    divided by the three products per algorithmic flop; every other kind (FP64
    arithmetic) against the cuBLAS FP64 GEMM rate measured in this run."""
    if kind == "apply" and precision == "tf32x3" and peaks.get("bf16_tflops"):
        return (peaks["bf16_tflops"] * TF32_PER_BF16 / 3.0, "tensor",
                f"TF32 dense = {src} BF16 x {TF32_PER_BF16:.3f} (nominal ratio), / 3 products per flop")
    return fp64, "alu", "cuBLAS FP64 GEMM 4096^3 measured in this run"


def main_full(args):
    """Alg. 2 step of the Hubbard L = 32 chain from a random full-rank iterate:
    every warm-up and timed step starts from the same iterate (uploaded before
    the timed region) with a fresh solver state, so the K timed steps are K
    passes of the same unit of work."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    prec = nat.PREC_TF32X3 if args.precision == "tf32x3" else nat.PREC_FP64
    ctx.set_jacobi_precond(args.jacobi_precond)
    S = setup(ctx, nat, seed=1)
    fl_branch = apply_flops_per_branch(nat, ctx, S)
    ctx.set_precision(prec)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    hx, bonds = S["x"].export(), S["x"].bonds()

    def fresh():
        return nat.mps_import(ctx, 32, 1, 16, 16, bonds, hx), nat.solver_state()

    def one_step(xx, state):
        return nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], state, xx)

    for _ in range(args.warmup):
        one_step(*fresh())
    ctx.sync()

    def timed_steps(profile):
        ms, fl, infos = 0.0, 0.0, []
        kinds = {}
        if profile:
            ctx.profile(True)
        for _ in range(args.steps):
            xx, state = fresh()
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = one_step(xx, state)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            fl += info["flops"]
            infos.append(info)
            if profile:
                for k, v in ctx.kernel_stats(reset=True).items():
                    a = kinds.setdefault(k, [0, 0.0, 0.0, 0.0])
                    for i in range(4):
                        a[i] += v[i]
        if profile:
            ctx.profile(False)
        return ms, fl, infos, kinds

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    total_ms, total_flops, infos, _ = timed_steps(False)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    from paper_2604_16118_gb300 import replicas
    total_ms, total_flops = replicas.reduce_timing(total_ms, total_flops, dist, dev)
    clocks = sampler.stop()
    # the same steps again, every launch bracketed by events
    prof_ms, _, prof_infos, kinds = timed_steps(True)
    apply_n, apply_ms, apply_fl, apply_by = kinds.get("apply", [0, 0.0, 0.0, 0.0])
    aq_n, aq_ms, aq_fl, _ = kinds.get("apply_qr", [0, 0.0, 0.0, 0.0])
    # the apply: contraction + the zip-up's own factorisation launches; its
    # algorithmic work is the contraction's (Sec. 2.4 work list)
    value = apply_fl / ((apply_ms + aq_ms) * 1e-3) / 1e12 if apply_ms else None
    contraction = apply_fl / (apply_ms * 1e-3) / 1e12 if apply_ms else None
    # end to end through the C ABI with host buffers: upload from pinned memory,
    # the step, the iterate read back
    pinned = torch.empty(len(hx), dtype=torch.float64).pin_memory()
    pinned.numpy()[:] = hx
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd = nat.mps_import(ctx, 32, 1, 16, 16, bonds, pinned.numpy())
        h2d += 8 * len(pinned)
        xd, info = one_step(xd, nat.solver_state())
        out_h = xd.export()
        d2h += 8 * len(out_h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_fl = apply_fl                    # the same steps as the profiled rerun
    peaks, src = measured_peaks()
    fp64 = fp64_gemm_peak(torch, dev)
    dom = max(kinds.items(), key=lambda kv: kv[1][1])
    dname, (dn, dms, dfl, dby) = dom
    dpeak, dbound, dsrc = kind_peak(dname, args.precision, fp64, peaks, src)
    apeak, abound, asrc = kind_peak("apply", args.precision, fp64, peaks, src)
    ach = dfl / (dms * 1e-3) / 1e12 if dms else None
    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64 (tf32x3 contraction)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one Alg. 2 step from the full-rank iterate (same input every step)",
                   "precision": args.precision, "jacobi_precond": args.jacobi_precond,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "value": "zip-up MPO application (all preconditioner branches): contraction flops / device "
                            "time of the contraction and the zip-up's factorisation launches, from the timed steps "
                            "rerun with per-launch events"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_fl / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps, "steps": args.steps,
                "what": "apply flops of the same steps / wall time of the steps through the C ABI with host "
                        "buffers (upload, step, download)"},
        "roofline": {"bound": dbound, "kernel": dname, "achieved": ach, "peak": dpeak, "unit": "TFLOP/s",
                     "frac": ach / dpeak if (ach and dpeak) else None, "traffic": None, "peak_source": dsrc,
                     "launches": dn, "kernel_ms": dms, "share": dms / sum(v[1] for v in kinds.values())},
        "apply": {"tflops": value, "ms": apply_ms + aq_ms, "flops": apply_fl,
                  "contraction": {"kernel": "k_gemm_tf32x3" if args.precision == "tf32x3" else "k_gemm/k_gemm_small",
                                  "launches": apply_n, "ms": apply_ms, "bytes": apply_by, "tflops": contraction,
                                  "peak": apeak, "bound": abound,
                                  "frac": contraction / apeak if (contraction and apeak) else None,
                                  "peak_source": asrc,
                                  "achieved_gbs": apply_by / (apply_ms * 1e-3) / 1e9 if apply_ms else None,
                                  "hbm_peak_gbs": peaks.get("hbm_gbs")},
                  "factorisation": {"launches": aq_n, "ms": aq_ms, "flops": aq_fl}},
        "step": {"ms": total_ms / args.steps, "tflops": total_flops / (total_ms * 1e-3) / 1e12,
                 "profiled_ms": prof_ms / args.steps},
        "kernels": {k: {"launches": v[0], "ms": v[1], "flops": v[2], "bytes": v[3]} for k, v in kinds.items()},
        "steps_info": [{"lambda": i["lambda"], "rho": i["rho"], "eta_tries": i["eta_tries"], "max_rank": i["max_rank"],
                        "flops": i["flops"], "precision": i["precision"]} for i in infos],
        "energy": infos[-1]["lambda"] - S["gamma"] if infos else None,
        "rerun_match": max(abs(a["rho"] - b["rho"]) for a, b in zip(infos, prof_infos)),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        reps = 10
        t1 = float(np.sum(oracle_apply_times(1, reps=reps)))
        tn = float(np.sum(oracle_apply_times(cores, reps=reps)))
        out["cpu_baseline"] = {"value": reps * fl_branch / t1 / 1e12, "unit": "TFLOP/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"{reps} oracle zip-up applications of one preconditioner branch of the "
                                         f"same rank-256 iterate ({t1:.1f} s on 1 core, numpy FP64)",
                               "all_cores": {"value": reps * fl_branch / tn / 1e12, "cores": cores, "seconds": tn,
                                             "what": "the same sample with BLAS on all host cores"}}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def main_tta(args):
    """Time to convergence of config 2 from e_1 (the paper's start, Sec. 7.1.4):
    Alg. 2 steps until rho^n <= 1e-8 (the residual bound of Eq. (rhobound)), the
    termination test holds, or the energy has settled at the rank cap (three
    consecutive changes below 1e-10 Eh), at most --max-steps steps and
    --max-seconds seconds; the precision of the contraction stage from
    --precision.  At r_max = 256 the cap's truncation error keeps rho far above
    1e-8, so the line also reports the time after which every energy stays
    within 1e-8 Eh of the last one (the fixed-rank limit, when the run settled)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    S = setup(ctx, nat, seed=None)
    ctx.set_precision(nat.PREC_TF32X3 if args.precision == "tf32x3" else nat.PREC_FP64)
    st = nat.solver_state()
    x = S["x"]
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    recs = []
    reached = None
    for n in range(args.max_steps):
        x, info = nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], st, x)
        el = time.perf_counter() - t0
        recs.append({"n": n, "t": el, "energy": info["lambda"] - S["gamma"], "rho": info["rho"],
                     "max_rank": info["max_rank"], "eta_tries": info["eta_tries"], "precision": info["precision"],
                     "flops": info["flops"]})
        if info["rho"] <= 1e-8 or info["converged"]:
            reached = el
            break
        if len(recs) >= 4 and all(abs(recs[-i]["energy"] - recs[-i - 1]["energy"]) < 1e-10 for i in (1, 2, 3)):
            break
        if el > args.max_seconds:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    settled = len(recs) >= 4 and all(abs(recs[-i]["energy"] - recs[-i - 1]["energy"]) < 1e-10 for i in (1, 2, 3))
    e_last = recs[-1]["energy"] if recs else None
    t_within = None
    for i in range(len(recs)):
        if all(abs(r["energy"] - e_last) <= 1e-8 for r in recs[i:]):
            t_within = recs[i]["t"]
            break
    out = {"metric": "time to residual bound rho <= 1e-8 (Alg. 2 from e_1)", "value": reached, "unit": "s",
           "time_to_1e-8_of_last": t_within if settled else None, "settled": settled,
           "n_gpus": 1, "steps": len(recs), "warmup": 0, "ms_per_step": 1e3 * wall / max(len(recs), 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f64 (tf32x3 contraction)", "data": "synthetic",
           "config": {"workload": WORKLOAD_E1.replace(", FP64", ""), "precision": args.precision,
                      "l2": "not flushed (one solve)"},
           "clocks": clocks, "wall_s": wall, "final_energy": recs[-1]["energy"] if recs else None,
           "split_steps": sum(1 for r in recs if r["precision"] != 0), "trajectory": recs,
           "e2e": {"value": reached, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main_tta_k12(args):
    """Time to |E - E_ref| <= 1e-8 on the spinless random chain K = 12, N = 6 of
    the config-1 generator (seed 0) from its random start of rank 32 (seed 0),
    without a rank cap (the cap of 32 leaves an error near 3e-4): Alg. 2 steps
    with the constants and the exact E_ref = lambda_1 - gamma stored by
    tests/golden/make_config1_trajectory.py; the contraction precision from
    --precision."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    from synth import random_block_values, spinless_random_chain
    with open(os.path.join(ROOT, "tests", "golden", "oracle_config1_trajectory.json")) as f:
        g = json.load(f)
    w, cst = g["workload"], g["constants"]
    wl = spinless_random_chain(K=w["K"], N=w["N"], seed=w["seed"])
    e_ref = cst["lambda1"] - cst["gamma"]
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, wl.n_up, cst["gamma"])
    p = nat.make_precond(np.array(cst["theta"]), cst["t_min"], cst["t_max"], cst["c0"], cst["alpha0"])
    sp = nat.solver_params(cst["c"], cst["delta"], eps_num=cst["eps_num"], t_eig=cst["t_eig"], tau=1e-12, r_max=0)
    vals = random_block_values(w["n_values"], w["seed"])
    ctx.set_precision(nat.PREC_TF32X3 if args.precision == "tf32x3" else nat.PREC_FP64)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x = nat.mps_create(ctx, wl.n_orb, 0, wl.n_up, 0, w["r_max"], vals)
    st = nat.solver_state()
    recs, reached = [], None
    for n in range(args.max_steps):
        x, info = nat.eigensolve_step(ctx, W, p, sp, st, x)
        el = time.perf_counter() - t0
        err = info["lambda"] - cst["gamma"] - e_ref
        recs.append({"n": n, "t": el, "error": err, "rho": info["rho"], "max_rank": info["max_rank"],
                     "precision": info["precision"]})
        if abs(err) <= 1e-8 and reached is None:
            reached = el
            break
        if info["converged"] or el > args.max_seconds:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    out = {"metric": "time to |E - E_ref| <= 1e-8 Eh (Alg. 2, exact E_ref)", "value": reached, "unit": "s",
           "n_gpus": 1, "steps": len(recs), "warmup": 0, "ms_per_step": 1e3 * wall / max(len(recs), 1),
           "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64 (tf32x3 contraction)",
           "data": "synthetic",
           "config": {"workload": "spinless_random_chain K=12 N=6 seed 0 (config-1 generator), random start of "
                                  "rank 32, no rank cap, constants and E_ref by exact diagonalisation",
                      "precision": args.precision, "l2": "not flushed (one solve)"},
           "clocks": clocks, "wall_s": wall, "final_error": recs[-1]["error"] if recs else None,
           "split_steps": sum(1 for r in recs if r["precision"] != 0), "trajectory": recs,
           "e2e": {"value": reached, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main_tta_learned(args):
    """Time to |E - E_ref| <= 1e-8 Eh on the spinless random chain K = 12, N = 6
    (config-1 generator, seed 0; E_ref exact, stored by
    tests/golden/make_config1_trajectory.py), from e_1 without a rank cap, in
    four arms: FP64 or split-precision (tf32x3) contraction, each with the plain
    preconditioner parameters (c_0 = 0.1, margin 1) or the learned controller's
    choice with its per-step plain fallback.  The controller is trained first,
    inside this run, on the plain solver's grid scores of 12 small problems
    (molecule-like L = 3, 4 and spinless chains K = 6, 8) by the library's
    tensor-core network kernels; its training time is reported separately.
    value: the mixed + learned arm's time; the plain FP64 arm's time beside it."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import learned as LP
    from paper_2604_16118_gb300 import native as nat
    from synth import molecule_like, spinless_random_chain
    with open(os.path.join(ROOT, "tests", "golden", "oracle_config1_trajectory.json")) as f:
        g = json.load(f)
    w, cst = g["workload"], g["constants"]
    e_ref = cst["lambda1"] - cst["gamma"]
    wl = spinless_random_chain(K=w["K"], N=w["N"], seed=w["seed"])
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    train_p = []
    for s_ in range(6):
        train_p.append(molecule_like(L=3 + s_ % 2, n_up=1 + s_ % 2, n_dn=1 + (s_ // 2) % 2, seed=100 + s_))
        K = 6 + 2 * (s_ % 2)
        train_p.append(spinless_random_chain(K=K, N=K // 2, seed=200 + s_))
    t0 = time.perf_counter()
    X, Y, _ = LP.make_dataset(ctx, train_p, n_steps=3)
    net, losses = LP.train(ctx, X, Y, steps=300)
    t_train = time.perf_counter() - t0
    choice = LP.choose(net, wl)
    sampler = ClockSampler(local)
    sampler.start()
    arms = {}
    for prec in ("fp64", "tf32x3"):
        for kind in ("plain", "learned"):
            ctx.set_precision(nat.PREC_TF32X3 if prec == "tf32x3" else nat.PREC_FP64)
            trace = []
            reached = []

            def stop(e):
                if abs(e - e_ref) <= 1e-8:
                    reached.append(True)
                    return True
                return False

            ctx.sync()
            E, F, used = LP.solve(ctx, net, wl, args.max_steps, r_max=0,
                                  params=LP.PLAIN if kind == "plain" else None, stop=stop, trace=trace)
            arms[f"{prec}+{kind}"] = {
                "seconds": trace[-1][0] if (trace and reached) else None, "steps": len(E),
                "final_error": E[-1] - e_ref if E else None, "gflop": sum(F) * 1e-9,
                "params": [list(u) for u in sorted(set(used))]}
    clocks = sampler.stop()
    ctx.set_precision(nat.PREC_FP64)
    ml, fp = arms["tf32x3+learned"]["seconds"], arms["fp64+plain"]["seconds"]
    out = {"metric": "time to |E - E_ref| <= 1e-8 Eh, mixed + learned vs FP64 plain", "value": ml, "unit": "s",
           "n_gpus": 1, "steps": arms["tf32x3+learned"]["steps"], "warmup": 0,
           "ms_per_step": 1e3 * ml / arms["tf32x3+learned"]["steps"] if ml else None,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (tf32x3 contraction)", "data": "synthetic",
           "config": {"workload": "spinless_random_chain K=12 N=6 seed 0 (config-1 generator) from e_1, no rank "
                                  "cap, E_ref by exact diagonalisation; set-up of the controller's problems "
                                  "(c = 0.7, delta = 20, t_eig = 0.5)",
                      "l2": "not flushed (one solve per arm)"},
           "clocks": clocks, "fp64_plain_seconds": fp, "speedup_vs_fp64_plain": (fp / ml) if (fp and ml) else None,
           "arms": arms, "controller": {"choice": list(choice), "train_seconds": t_train,
                                        "loss_first_last": [losses[0], losses[-1]], "samples": int(len(X))},
           "e2e": {"value": ml, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main_batched(args):
    """The batched form: zip-up applications of 128 independent molecule-like
    Hamiltonians (the generator of configs 3 and 4; L cycling through 3..6,
    N = L, ranks cycling through 64, 128, 256, 512, capped by the exact ranks;
    seeds 1000 + i) in one batched call, against one call per instance.  Each is
    timed with events on the library's stream after a warm-up (which also fixes
    the contraction autotuner's choices), L2 flushed before every repetition."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build, problem
    build.build()
    from paper_2604_16118_gb300 import native as nat
    from synth import molecule_like, random_block_values
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    n_inst = 128
    Ls, ranks = (3, 4, 5, 6), (64, 128, 256, 512)
    Ws, xs, shifts, shapes = [], [], [], []
    for i in range(n_inst):
        L, r = Ls[i % 4], ranks[(i // 4) % 4]
        wl = molecule_like(L=L, n_up=(L + 1) // 2, n_dn=L // 2, seed=1000 + i)
        gamma = problem.cholesky_shift(wl.h, wl.eri, wl.n_up, wl.n_dn, 1, margin=1.0)
        nval = nat.mps_random_size(L, 1, wl.n_up, wl.n_dn, r)
        xs.append(nat.mps_create(ctx, L, 1, wl.n_up, wl.n_dn, r, random_block_values(nval, 1000 + i)))
        Ws.append(nat.mpo_from_integrals(ctx, wl.h, wl.eri, 1, wl.n_particles, gamma))
        shifts.append(-1.0)
        shapes.append((L, r, max(xs[-1].ranks())))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        ms = []
        for it in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            del out
            if it >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    ys, fl = nat.apply_zipup_batch(ctx, Ws, xs, shifts)
    l0 = ctx.launch_count()
    ms_batch = timed(lambda: nat.apply_zipup_batch(ctx, Ws, xs, shifts))
    lb = (ctx.launch_count() - l0) // (args.warmup + args.steps)
    l0 = ctx.launch_count()
    ms_single = timed(lambda: [nat.apply_zipup(ctx, W, x, s) for W, x, s in zip(Ws, xs, shifts)])
    ls = (ctx.launch_count() - l0) // (args.warmup + args.steps)
    # the batch recorded once as a CUDA graph, replayed
    plan = nat.ZipupPlan(ctx, Ws, xs, shifts)
    l0 = ctx.launch_count()
    ms_graph = timed(lambda: plan.launch())
    lg = (ctx.launch_count() - l0) // (args.warmup + args.steps)
    ctx.sync()
    graph_diff = max(float(np.abs(a.export() - b.export()).max() / max(np.abs(b.export()).max(), 1e-300))
                     for a, b in zip(plan.outputs, ys))
    # end to end: the iterates' values uploaded from pinned host memory, one graph
    # launch, the outputs read back
    host_x = [torch.from_numpy(x.export()).pin_memory() for x in xs]
    h2d = sum(8 * v.numel() for v in host_x)
    d2h = sum(8 * y.size() for y in plan.outputs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for x, v in zip(xs, host_x):
            x.write(v.numpy())
        plan.launch()
        for y in plan.outputs:
            y.export()
    e2e_s = (time.perf_counter() - t0) / args.steps
    tf = lambda ms: fl / (ms * 1e-3) / 1e12
    out = {"metric": "MPO.MPS apply, 128 independent Hamiltonians, TFLOP/s", "value": tf(ms_graph),
           "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "128 molecule-like Hamiltonians (L cycling 3..6, N = L, r cycling 64..512 capped "
                                  "by the exact ranks), zip-up application of a random iterate each",
                      "l2": "flushed before every repetition",
                      "value": "the batch recorded as one CUDA graph (bsmps_plan_apply_zipup_batch), replayed"},
           "gpu_launches": lg,
           "graph": {"ms": ms_graph, "launches": lg, "tflops": tf(ms_graph), "max_rel_diff_vs_batched": graph_diff},
           "batched": {"ms": ms_batch, "launches": lb, "tflops": tf(ms_batch)},
           "one_by_one": {"ms": ms_single, "launches": ls, "tflops": tf(ms_single)},
           "speedup_graph_vs_one_by_one": ms_single / ms_graph, "speedup_batched_vs_one_by_one": ms_single / ms_batch,
           "flops": fl, "max_ranks": sorted(set(s[2] for s in shapes)),
           "e2e": {"value": fl / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h,
                   "what": "bsmps_mps_write of every iterate from pinned host memory, one graph launch, "
                           "bsmps_mps_export of every output"}}
    print(json.dumps(out))
    return 0


def main_mlp(args):
    """Training steps of the learned controller's network (128 -> 256 -> 256 ->
    256 -> 2, BF16 weights, FP32 accumulation) on a synthetic batch of 8192:
    forward, backward and Adam per step, every product on the tensor cores
    (tcgen05 kind::tf32).  value: the products' FP32 flops over their device
    time (CUDA events around each product launch, the library's profiler); the
    step's wall time (batch upload, loss read-back) beside it."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    stream = torch.cuda.Stream(device=dev)
    ctx = nat.Context(local, stream.cuda_stream)
    widths = [128, 256, 256, 256, 2]
    rng = np.random.default_rng(0)
    n_par = sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1))
    parts = []
    for i in range(len(widths) - 1):
        parts.append(rng.standard_normal(widths[i] * widths[i + 1]) * np.sqrt(2.0 / widths[i]))
        parts.append(np.zeros(widths[i + 1]))
    p0 = np.concatenate(parts).astype(np.float32)
    assert len(p0) == n_par
    B = 8192
    x = rng.standard_normal((B, 128)).astype(np.float32)
    t = np.tanh(x @ (rng.standard_normal((128, 2)).astype(np.float32) / 12.0))
    net = nat.MLP(ctx, widths, p0)
    for _ in range(args.warmup):
        net.train_step(x, t, 1e-3)
    ctx.sync()
    ctx.kernel_stats(reset=True)
    ctx.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = [net.train_step(x, t, 1e-3) for _ in range(args.steps)]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    ctx.profile(False)
    n, ms, fl, by = ctx.kernel_stats(reset=True)["mlp"]
    peaks, src = measured_peaks()
    tf32_peak = peaks["bf16_tflops"] * TF32_PER_BF16 if peaks.get("bf16_tflops") else None
    ach = fl / (ms * 1e-3) / 1e12 if ms else None
    out = {"metric": "learned-controller network training, tensor-core products", "value": ach, "unit": "TFLOP/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32 (bf16 weights)",
           "data": "synthetic",
           "config": {"workload": f"MLP {widths}, batch {B}, forward + backward + Adam per step",
                      "l2": "not flushed (the working set is L2-resident by design)"},
           "gpu_launches": n, "clocks": clocks,
           "roofline": {"bound": "tensor", "kernel": "k_mlp_gemm_tc", "achieved": ach, "peak": tf32_peak,
                        "unit": "TFLOP/s", "frac": ach / tf32_peak if (ach and tf32_peak) else None,
                        "traffic": None,
                        "peak_source": f"TF32 dense = {src} BF16 x {TF32_PER_BF16:.3f} (nominal ratio)"},
           "products": {"launches": n, "ms": ms, "flops": fl}, "loss_first_last": [losses[0], losses[-1]],
           "e2e": {"value": fl / wall / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 4 * (x.size + t.size),
                   "d2h_bytes_per_step": 4 * B * 2}}
    print(json.dumps(out))
    return 0


def main_profile(args):
    """Small fixed runs for profilers (no timing of their own):
    profile_step: one Alg. 2 step of the default workload (Hubbard L = 32 from the
    seed-1 rank-256 iterate); profile_apply: the zip-up application of that
    iterate, twice; profile_truncation: one truncation of a random spinless
    K = 20, N = 10 iterate at exact ranks (sectors up to 252 wide).
    --precision selects the contraction arithmetic."""
    from paper_2604_16118_gb300 import build
    build.build()
    from paper_2604_16118_gb300 import native as nat
    ctx = nat.Context(0)
    ctx.set_precision(nat.PREC_TF32X3 if args.precision == "tf32x3" else nat.PREC_FP64)
    ctx.set_jacobi_precond(args.jacobi_precond)
    t0 = time.perf_counter()
    if args.workload == "profile_truncation":
        from synth import random_block_values
        n = nat.mps_random_size(20, 0, 10, 0, 1024)
        x = nat.mps_create(ctx, 20, 0, 10, 0, 1024, random_block_values(n, 7))
        z, _, _ = nat.truncate(ctx, x, 1e-3)
        what = {"max_rank": max(z.ranks())}
    else:
        S = setup(ctx, nat, seed=1)
        if args.workload == "profile_apply":
            for _ in range(2):
                y, fl = nat.apply_zipup(ctx, S["W"], S["x"], shift=-70.0)
            what = {"flops": fl, "max_rank": max(y.ranks())}
        else:
            _, info = nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], nat.solver_state(), S["x"])
            what = {"lambda": info["lambda"], "rho": info["rho"], "flops": info["flops"]}
    ctx.sync()
    print(json.dumps({"workload": args.workload, "precision": args.precision, "jacobi_precond": args.jacobi_precond,
                      "wall_s": time.perf_counter() - t0,
                      **what}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "tf32x3"],
                    help="arithmetic of the zip-up contraction stage")
    ap.add_argument("--jacobi-precond", type=int, default=48,
                    help="truncation SVDs with k >= this start from an FP32 Jacobi (0: never)")
    ap.add_argument("--max-steps", type=int, default=400, help="hubbard_tta: step limit")
    ap.add_argument("--max-seconds", type=float, default=1800.0, help="hubbard_tta: time limit")
    ap.add_argument("--workload", default="hubbard",
                    choices=["hubbard", "hubbard_e1", "hubbard_tta", "tta_k12", "tta_learned", "batched",
                             "coulomb14_alg4_D4",
                             "coulomb14_alg3", "ozaki_gemm", "mlp", "profile_step", "profile_apply",
                             "profile_truncation"],
                    help="hubbard: Alg. 2 steps at full rank (the JSON contract); hubbard_e1: the trajectory "
                         "from e_1; hubbard_tta: time to convergence from e_1; coulomb14_alg4_D4: Alg. 4 (D = 4); "
                         "coulomb14_alg3: time to solution of the paper's K = 14 run; "
                         "ozaki_gemm: the emulated FP64 GEMM vs DGEMM")
    args = ap.parse_args()
    if args.workload == "coulomb14_alg3":
        return main_outer(args)
    if args.workload == "coulomb14_alg4_D4":
        return main_joint(args)
    if args.workload == "ozaki_gemm":
        return main_ozaki(args)
    if args.workload == "hubbard_tta":
        return main_tta(args)
    if args.workload == "tta_k12":
        return main_tta_k12(args)
    if args.workload == "tta_learned":
        return main_tta_learned(args)
    if args.workload == "batched":
        return main_batched(args)
    if args.workload == "mlp":
        return main_mlp(args)
    if args.workload.startswith("profile_"):
        return main_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "hubbard_e1":
        return main_e1(args)
    return main_full(args)


if __name__ == "__main__":
    sys.exit(main())
