#!/usr/bin/env python
"""Benchmark of the GB300 DMRG hot path.

Workload: pf shell, 40 m-scheme sites, 8 protons + 8 neutrons, M_z = 0 (m-scheme
dimension 1,087,455,228), J-coupled random two-body ensemble (sigma = 1 MeV, seed 3),
single-particle energies U[0,4) MeV, M = 4096 block states.  Setup (untimed): starting
state with M = 4096 per right block, block build, two-site steps from position 1 to the
middle of the chain.  A timed step is one full two-site DMRG step at the middle of the
chain (superblock operators, Davidson with H_eff products, reduced-density-matrix
truncation, renormalization of every normal and complementary operator) in the mixed
path (FP32 operator contractions, FP64 Davidson / eigensolver / energy).

Reported: value = H_eff psi TFLOP/s over the timed steps (algorithmic flops of every
H_eff product / device time of the whole steps, CUDA events), the H_eff products' own
device time and their HBM roofline, the FP64 path on the same superblock and the energy
difference between the two, e2e = the same metric over a whole job through the public API
(fresh context from host arrays, block build, one sweep at M = 4096 from the starting
state, energy read back; wall clock), sweep_s = that sweep's seconds, a batch of 32
small instances looped vs batched, and the FP64 CPU oracle as the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff·ψ TFLOP/s + sweep s at M=4096, mixed vs FP64 GPU at |ΔE|≤1e-5 MeV"
WORKLOAD = dict(space="pf", Np=8, Nn=8, two_Mz=0, seed=3, mps_seed=3003, M=4096)
WORKLOAD_NAME = ("pf-shell 40 sites, 8p+8n, M_z=0 (m-scheme dim 1,087,455,228), random "
                 "J-coupled TBME sigma=1 MeV seed 3, M=4096, mid-chain two-site steps")
# DRAM bytes (read + write) per mixed H_eff product of the default workload, from the one-pass
# ncu capture of the timed steps in profiles/step_kernels_pf8p8n_M4096.md (sum over the
# product's kernels / products); to be re-taken whenever those kernels change
HEFF_TRAFFIC_BYTES = 175.3e6
CPU_SAMPLE = dict(space="sd", Np=2, Nn=2, two_Mz=0, seed=1, mps_seed=5, M=64)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = str(gpu_index)
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[0] == self.idx:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _positions(N, start, count):
    """(p, dir) of a sweep starting at `start` left to right, then back."""
    seq = [(p, 0) for p in range(1, N - 2)] + [(p, 1) for p in range(N - 3, 0, -1)]
    i = [x for x, (p, d) in enumerate(seq) if p == start and d == 0][0]
    out = []
    while len(out) < count:
        out.append(seq[i % len(seq)])
        i += 1
    return seq[:[x for x, (p, d) in enumerate(seq) if p == start and d == 0][0]], out


# ------------------------------------------------------------------------------------
# CPU oracle sample (FP64, numpy, one thread): H_eff products inside two-site steps
# ------------------------------------------------------------------------------------
def _oracle_heff_flops(sb):
    idx = sb.layout.index()
    f = 0.0
    for Lk, Rk in zip(sb.L.ops, sb.R.ops):
        for (QLo, QLi), Lb in Lk.items():
            if QLi not in idx or QLo not in idx:
                continue
            _, QRi, dLi, dRi, _ = idx[QLi]
            _, QRo, dLo, dRo, _ = idx[QLo]
            if (QRo, QRi) not in Rk:
                continue
            f1 = 2.0 * dLi * dRi * dRo + 2.0 * dLo * dLi * dRo
            f2 = 2.0 * dLo * dLi * dRi + 2.0 * dLo * dRi * dRo
            f += min(f1, f2)
    return f


def cpu_oracle_sample(steps, warmup, budget_s=25.0):
    """Times the oracle's H_eff products during two-site steps of the sd 2p+2n, M=64
    workload (FP64 numpy).  Returns (TFLOP/s, seconds, products, description)."""
    from gen import make_problem, initial_mps
    from oracle.dmrg import OracleDMRG
    w = CPU_SAMPLE
    prob = make_problem(w["space"], w["Np"], w["Nn"], w["two_Mz"], seed=w["seed"])
    o = OracleDMRG(prob, initial_mps(prob, w["M"], w["mps_seed"]))
    # instrument the oracle's superblock product (timing only; arithmetic untouched)
    stats = {"flops": 0.0, "t": 0.0, "n": 0}
    orig = o.superblock

    def timed_superblock(p):
        sb = orig(p)
        fl = _oracle_heff_flops(sb)
        app = sb.apply

        def apply(x):
            t0 = time.perf_counter()
            y = app(x)
            stats["t"] += time.perf_counter() - t0
            stats["flops"] += fl
            stats["n"] += 1
            return y
        sb.apply = apply
        return sb
    o.superblock = timed_superblock
    N = prob.n_sites
    mid = N // 2 - 1
    t_start = time.perf_counter()
    for p in range(1, mid):
        o.run_step(p, "L", w["M"])
    stats.update(flops=0.0, t=0.0, n=0)
    done = 0
    for p in range(mid, N - 2):
        if done >= warmup + steps or time.perf_counter() - t_start > budget_s:
            break
        if done == warmup:
            stats.update(flops=0.0, t=0.0, n=0)
        o.run_step(p, "L", w["M"])
        done += 1
    tf = stats["flops"] / max(stats["t"], 1e-12) / 1e12
    desc = (f"oracle H_eff products in {max(done - warmup, 0)} mid-chain two-site steps of sd "
            f"2p+2n (m-scheme dim 640), M=64, FP64 numpy; {stats['n']} products, "
            f"{stats['t']:.2f} s (the pf 8p+8n environment takes the plain oracle ~200 s to "
            f"build)")
    return tf, stats["t"], stats["n"], desc


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    tf, secs, nprod, desc = cpu_oracle_sample(args.steps, args.warmup, budget_s=240.0)
    line = {"impl": "reference", "metric": METRIC, "value": tf, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample": desc},
            "cpu_baseline": {"value": tf, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": tf, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_baseline_subprocess(steps, warmup):
    """The oracle sample in a child process pinned to one BLAS thread."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_sample(%d, %d)))" % (ROOT, steps, warmup))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        return None
    tf, secs, nprod, desc = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": tf, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": desc,
            "host_cores": os.cpu_count()}


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------
def batch_instances(M_cap):
    """Batch workload: 32 instances, even i -> sd, odd i -> pf; N_p = 2 + (7 i mod 9),
    N_n = 2 + (5 i mod 9) capped at the space; M = 128 * 2^(i mod 5) capped; seeds 1000+i."""
    from gen import make_problem, SPACES
    out = []
    for i in range(32):
        space = "sd" if i % 2 == 0 else "pf"
        cap = SPACES[space].states_per_species - 2
        Np = min(2 + (7 * i) % 9, cap)
        Nn = min(2 + (5 * i) % 9, cap)
        M = min(128 * 2 ** (i % 5), M_cap)
        out.append((make_problem(space, Np, Nn, (Np + Nn) % 2, seed=1000 + i), M, 2000 + i))
    return out


def run_batch_compare(P, M_cap):
    """One sweep of every instance: looped one context at a time, then as one batch."""
    import torch
    from gen import initial_mps
    inst = batch_instances(M_cap)
    inits = [initial_mps(prob, M, s) for prob, M, s in inst]

    streams = [torch.cuda.Stream() for _ in inst]   # one stream per instance

    def make():
        ds = []
        for (prob, M, s), init, st in zip(inst, inits, streams):
            d = P.DMRG(prob, precision=P.MIXED_FP32, stream=st)
            d.build_blocks(init)
            ds.append(d)
        return ds
    loop = make()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_loop = [d.sweep(M)[1] for d, (_, M, _) in zip(loop, inst)]
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    cs = [d.counters() for d in loop]
    loop_phases = {k: sum(c[k] for c in cs) for k in ("t_super", "t_enlarge", "t_davidson",
                                                      "t_truncate", "t_sync", "pool_mallocs")}
    loop_phases["t_malloc"] = cs[-1]["t_detail"][15]
    loop_phases["t_dav_host"] = sum(c["t_detail"][17] for c in cs)
    loop_phases["steps"] = sum(2 * (prob.n_sites - 3) for prob, _, _ in inst)
    bat = make()
    b = P.Batch(bat)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_bat, st = b.sweep([M for _, M, _ in inst])
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    dE = max(abs(a - c) for a, c in zip(e_loop, e_bat))
    b.close()
    return {"instances": len(inst), "M_cap": M_cap, "loop_sweep_s": t_loop,
            "batch_sweep_s": t_bat, "speedup": t_loop / t_bat,
            "batched_products": st["products"], "batched_heff_device_s": st["heff_seconds"],
            "max_dE_batch_vs_loop": dE, "loop_phase_s": loop_phases,
            "workload": "32 instances: even i sd, odd i pf, N_p=2+(7i mod 9), N_n=2+(5i mod 9), "
                        "M=128*2^(i mod 5) capped at %d, seeds 1000+i, mixed path" % M_cap}


def run_precond_compare(P):
    """Learned vs diagonal Davidson preconditioner: harvest two sweeps of sd 4p+4n at
    M = 256, train the network on the GPU (20 epochs), then Davidson from the uniform guess at every
    position of one sweep with each preconditioner (same converged energies)."""
    import torch
    from gen import make_problem, initial_mps
    prob = make_problem("sd", 4, 4, 0, seed=1)
    d = P.DMRG(prob, precision=P.MIXED_FP32)
    d.build_blocks(initial_mps(prob, 256, 5))
    t0 = time.perf_counter()
    d.mlp_harvest(True, 2048)
    d.sweep(256)
    d.sweep(256)
    d.mlp_harvest(False)
    d.mlp_reset(3)
    loss0, ns = d.mlp_train(epochs=1, batch=1024, lr=1e-3, seed=3)
    loss1, _ = d.mlp_train(epochs=20, batch=1024, lr=1e-3, seed=4)
    t_train = time.perf_counter() - t0
    n_diag = n_mlp = 0
    dmax = 0.0
    N = prob.n_sites
    for p in range(1, N - 2):
        size = d.psi_layout(p)["size"]
        x0 = torch.ones(size, dtype=torch.float64, device="cuda")
        d.set_options(precision=P.MIXED_FP32, precond=P.PRECOND_DIAG)
        e1, s1 = d.davidson(p, guess=x0, allow_noconv=True)
        d.set_options(precision=P.MIXED_FP32, precond=P.PRECOND_MLP)
        e2, s2 = d.davidson(p, guess=x0, allow_noconv=True)
        n_diag += s1["n_products"]
        n_mlp += s2["n_products"]
        dmax = max(dmax, abs(e1 - e2))
        d.set_options(precision=P.MIXED_FP32, precond=P.PRECOND_DIAG)
        d.step(p, 0, 256)
    d.close()
    return {"workload": "sd 4p+4n seed 1, M=256, two harvested sweeps, 20 epochs; Davidson from "
                        "the uniform guess at positions 1..%d, mixed path" % (N - 3),
            "samples": ns, "loss": [loss0, loss1], "train_s": t_train,
            "products_diagonal": n_diag, "products_learned": n_mlp,
            "max_dE": dmax}


def run_next_rows(P, prob, init, M, e_fixed):
    """Rows beyond the core path, each timed once by wall clock around a whole sweep:
    dynamic block state selection on the default workload (mixed path, M_min = 256,
    ceiling M, discarded-weight target 1e-5; compared with the fixed-M sweep from the same
    starting state), and two-state targeting on pf 4p+4n at M = 1024 in FP64 (one state
    vs the two lowest, from the same starting state)."""
    import torch
    from gen import make_problem, initial_mps
    out = {}
    try:
        d = P.DMRG(prob, precision=P.MIXED_FP32, dav_tol=1e-8)
        d.build_blocks(init)
        d.set_dbss(256, 1e-5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, e = d.sweep(M)
        torch.cuda.synchronize()
        kept = [s["kept"] for s in steps]
        out["dbss"] = {"workload": "default workload, M_min=256, M_max=%d, target 1e-5, one "
                                   "sweep from the starting state, mixed path" % M,
                       "sweep_s": time.perf_counter() - t0, "energy": e,
                       "dE_vs_fixed_M": e - e_fixed if e_fixed is not None else None,
                       "kept_min": min(kept), "kept_max": max(kept),
                       "kept_mean": sum(kept) / len(kept),
                       "trunc_err_max": max(s["trunc_err"] for s in steps),
                       "products": sum(s["n_products"] for s in steps)}
        d.close()
    except Exception as exc:          # a side measurement never takes the bench line down
        out["dbss"] = {"error": str(exc)}
    try:
        prob2 = make_problem("pf", 4, 4, 0, seed=2)
        init2 = initial_mps(prob2, 1024, 2002)
        res = {}
        for n_roots in (1, 2):
            d = P.DMRG(prob2, precision=P.FP64, dav_tol=1e-8)
            d.build_blocks(init2)
            d.set_roots(n_roots)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps, _ = d.sweep(1024)
            torch.cuda.synchronize()
            res[n_roots] = (time.perf_counter() - t0, steps)
            d.close()
        s1, s2 = res[1][1], res[2][1]
        out["two_state"] = {"workload": "pf 4p+4n seed 2, M=1024, FP64, one sweep from the "
                                        "same starting state",
                            "one_state_sweep_s": res[1][0], "two_state_sweep_s": res[2][0],
                            "products_one": sum(s["n_products"] for s in s1),
                            "products_two": sum(s["n_products"] for s in s2),
                            "E0": s2[-1]["energy"], "E1": s2[-1]["energy1"],
                            "excitation": s2[-1]["energy1"] - s2[-1]["energy"],
                            "E0_one_state": s1[-1]["energy"]}
    except Exception as exc:
        out["two_state"] = {"error": str(exc)}
    return out


def max_over_ranks(x, dist=None):
    """The largest value of x over the ranks of the process group (x on a single rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, flops_per_rank, seconds_max):
    """Whole-job TFLOP/s of `world` replicas: the work of every rank over the time of the
    slowest one."""
    return world * flops_per_rank / seconds_max / 1e12


def run_gpu(args):
    import ctypes
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_1507_00161_gb300.build import build
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    import paper_1507_00161_gb300 as P
    from gen import make_problem, initial_mps
    w = dict(WORKLOAD)
    wname = WORKLOAD_NAME
    if args.workload:
        # another system of the same family (profiling of smaller cases)
        sp, npr, nne, sd = args.workload.split(":")
        w.update(space=sp, Np=int(npr), Nn=int(nne), seed=int(sd), two_Mz=(int(npr) + int(nne)) % 2)
        wname = "%s shell, %dp+%dn, seed %d, M=%d (profiling case)" % (sp, int(npr), int(nne),
                                                                       int(sd), args.M)
    M = args.M
    prob = make_problem(w["space"], w["Np"], w["Nn"], w["two_Mz"], seed=w["seed"])
    init = initial_mps(prob, M, w["mps_seed"])
    d = P.DMRG(prob, precision=P.MIXED_FP32, dav_tol=1e-8, dav_max_iter=args.max_iter)
    d.build_blocks(init)
    N = prob.n_sites
    start = N // 2 - 1 - args.warmup
    setup, seq = _positions(N, max(start, 1), args.warmup + args.steps)
    for (p, dr) in setup:
        d.step(p, dr, M)
    for (p, dr) in seq[:args.warmup]:
        d.step(p, dr, M)
    timed = seq[args.warmup:]
    torch.cuda.synchronize()
    c0 = d.counters()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(timed) + 1)]
    stats = []
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if args.profile_range:
            torch.cuda.profiler.start()
        ev[0].record()
        for i, (p, dr) in enumerate(timed):
            stats.append(d.step(p, dr, M))
            ev[i + 1].record()
        torch.cuda.synchronize()
        if args.profile_range:
            torch.cuda.profiler.stop()
        if dist:
            dist.barrier()
    c1 = d.counters()
    free_b, total_b = torch.cuda.mem_get_info()
    dev_used_gb = (total_b - free_b) / 1e9
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(timed))]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, dist)
    flops = sum(s["heff_flops"] * s["n_products"] for s in stats)
    heff_s = sum(s["heff_seconds"] for s in stats)
    heff_bytes = sum(s["heff_bytes"] * s["n_products"] for s in stats)
    nprod = sum(s["n_products"] for s in stats)
    value = replica_throughput(world, flops, total_s)
    peak, peak_kind = _peaks()
    achieved = heff_bytes / max(heff_s, 1e-12) / 1e9
    p_e2e, _ = seq[-1]
    # dot-orbital density matrix of the last timed step's wave function (wall clock of the
    # whole call: piece lists on the host, two kernels, read-back)
    dot = None
    try:
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ent = d.dot_rdm(p_e2e)
            ts.append(time.perf_counter() - t0)
        size_last = d.psi_layout(p_e2e)["size"]
        dot = {"position": p_e2e, "wall_ms": 1e3 * min(ts), "psi_elements": size_last,
               "s_p": ent[0], "s_p1": ent[1], "I": ent[3]}
    except Exception as exc:
        dot = {"error": str(exc)}
    lay = d.psi_layout(p_e2e)
    # FP64 path on the same superblock: Davidson from the mixed eigenvector
    psi_m = torch.empty(lay["size"], dtype=torch.float64, device="cuda")
    e_mixed, st_m = d.davidson(p_e2e, out=psi_m, allow_noconv=True)
    d.set_options(precision=P.FP64, dav_tol=1e-8, dav_max_iter=args.max_iter)
    c2 = d.counters()
    e_fp64, st_d = d.davidson(p_e2e, guess=psi_m, allow_noconv=True)
    c3 = d.counters()
    fp64_tf = (c3["heff_flops"] - c2["heff_flops"]) / max(c3["heff_seconds"] - c2["heff_seconds"],
                                                           1e-12) / 1e12
    d.set_options(precision=P.MIXED_FP32, dav_tol=1e-8, dav_max_iter=args.max_iter)
    d.close()
    del d
    # end to end through the public API: a fresh context from the host arrays of the
    # Hamiltonian and the starting state (copied to the device inside the timed region),
    # the block build, one full sweep at M, the energy read back to the host
    e2e = None
    sweep_s = None
    if args.sweep:
        h2d = sum(int(a.nbytes) for a in (prob.species, prob.two_m, prob.eps, prob.v_idx,
                                          prob.v_val, prob.order))
        h2d += sum(int(np.asarray(a).nbytes) for a in init.flat())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dj = P.DMRG(prob, precision=P.MIXED_FP32, dav_tol=1e-8, dav_max_iter=args.max_iter)
        dj.build_blocks(init)
        t1 = time.perf_counter()
        sw_steps, e_sweep = dj.sweep(M)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        sweep_s = t2 - t1
        sw_flops = sum(s["heff_flops"] * s["n_products"] for s in sw_steps)
        e2e = {"value": sw_flops / (t2 - t0) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8 + len(sw_steps) * ctypes.sizeof(P.StepStats),
               "job": "create from host arrays + block build + one sweep (%d steps, %d H_eff "
                      "products) + energy read back; wall clock" % (len(sw_steps),
                      sum(s["n_products"] for s in sw_steps)),
               "build_s": t1 - t0, "sweep_energy": e_sweep}
        dj.close()
        del dj
    clocks = clk.summary()
    batch = None
    if args.batch_mcap > 0:
        batch = run_batch_compare(P, args.batch_mcap)
    precond = run_precond_compare(P) if args.precond else None
    next_rows = None
    if args.next_rows:
        next_rows = run_next_rows(P, prob, init, M, e2e["sweep_energy"] if e2e else None)
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = _cpu_baseline_subprocess(args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wname, "M": M, "positions": timed,
                   "precision": "FP32 contractions, FP64 Davidson/eigensolver/energy",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2: %.0f MB of operator blocks per H_eff product"
                         % (heff_bytes / max(nprod, 1) / 1e6)},
        "heff": {"tflops_device": flops / max(heff_s, 1e-12) / 1e12, "products": nprod,
                 "device_s": heff_s, "flops_per_product": flops / max(nprod, 1),
                 "bytes_per_product": heff_bytes / max(nprod, 1)},
        "sweep_s": sweep_s,
        "fp64": {"heff_tflops": fp64_tf, "energy": e_fp64, "products": st_d["n_products"],
                 "energy_mixed": e_mixed, "dE_mixed_vs_fp64": abs(e_mixed - e_fp64)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": HEFF_TRAFFIC_BYTES if not args.workload and M == WORKLOAD["M"]
                     else None,
                     "kernel": "H_eff product: k_pad_psi + k_heff_small + k_heff_tc + k_heff_reduce + k_to_f64, CUDA events on the context stream around each product",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "batch": batch,
        "precond": precond,
        "next_rows": next_rows,
        "dot_rdm": dot,
        "e2e": e2e,
        "gpu_launches": int(c1["launches"] - c0["launches"]),
        "device_mem_used_gb": dev_used_gb,
        "phase_s": {k: c1[k] - c0[k] for k in ("t_enlarge", "t_super", "t_davidson",
                                               "t_truncate", "t_project", "t_predict",
                                               "t_sync", "t_enlarge_host", "t_upload")},
        "upload_bytes": c1["upload_bytes"] - c0["upload_bytes"],
        "pool_mallocs": c1["pool_mallocs"] - c0["pool_mallocs"],
        "host_detail_s": [b - a for a, b in zip(c0["t_detail"], c1["t_detail"])],
        "superblock": {k: c1[k] for k in ("sb_blocks_l", "sb_blocks_r", "sb_terms", "sb_tiles",
                                           "sb_small_tiles", "sb_term_hist",
                                           "sb_kernel_flops")},
        "clocks": clocks,
        "energies": [s["energy"] for s in stats],
        "step_ms": step_ms,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--M", type=int, default=WORKLOAD["M"])
    ap.add_argument("--max-iter", type=int, default=100)
    ap.add_argument("--sweep", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-mcap", type=int, default=256,
                    help="M cap of the 32-instance batch-vs-loop comparison (0: skip)")
    ap.add_argument("--precond", type=int, default=1,
                    help="learned vs diagonal preconditioner comparison (0: skip)")
    ap.add_argument("--next-rows", type=int, default=1,
                    help="also time a DBSS sweep and a two-state sweep (side measurements)")
    ap.add_argument("--workload", default="",
                    help="space:Np:Nn:seed of another system (profiling of smaller cases)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
