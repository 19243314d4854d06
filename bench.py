#!/usr/bin/env python
"""Benchmark of the GB300 DMRG hot path.

Workload (the headline configuration): pf shell, 40 m-scheme sites, 8 protons + 8 neutrons,
M_z = 0 (m-scheme dimension 1,087,455,228), J-coupled random two-body ensemble (sigma = 1
MeV, seed 3), single-particle energies U[0,4) MeV; seeded random starting state (seed
3003); M schedule 512(2) -> 1024(2) -> 2048(2) -> 4096(4) sweeps.

* e2e: the whole schedule as one job through the public API: a context created from the
  host arrays of the Hamiltonian, the blocks built from the host starting state, ten
  sweeps, every sweep's step records and energy read back; H_eff TFLOP/s over the job's
  wall clock.  The sweeps at M = 4096 give sweep_s (median, CUDA events).
* value: H_eff TFLOP/s over K two-site steps at M = 4096 after the schedule (left to
  right, centred on the middle of the chain, after W warm-up steps): algorithmic flops of
  every H_eff product / device time of the whole steps (superblock operators, Davidson,
  truncation by the density-matrix SVDs, renormalization of every normal and complementary
  operator), mixed path: FP32 operator contractions on split-TF32 tensor cores, FP64
  Davidson vectors, SVDs and energies.
* roofline: the H_eff product's algorithmic bytes / its device time (CUDA events around
  every product) against the measured copy bandwidth.
* fp64: mixed vs FP64 Davidson on the identical superblock of the heaviest timed position
  (the energy gate), and one FP64 sweep at M = 4096 from the state the schedule reached.
* cpu_baseline: the FP64 oracle's H_eff products on the same workload (position 1), timed
  on the host cores in a child process.
Side measurements (the schedule's sweeps, the timed steps, batch mode, the learned
preconditioner, the next rows, the pf+g9/2 12p+12n workload at 2M_z = 0 and 4) are printed
on lines of their own before the final line.

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
                 "J-coupled TBME sigma=1 MeV seed 3, schedule 512(2)->1024(2)->2048(2)->"
                 "4096(4), then two-site steps at M=4096 centred on the middle of the chain")
# the oracle's sample of the same workload: its H_eff products at position 1 with the
# starting state's right blocks at M0 states (building those blocks is not timed)
CPU_SAMPLE_M0 = 256
# DRAM bytes (read + write, ncu dram__bytes_read/write.sum) of the mixed product's kernels
# per algorithmic byte: 137.4 MB against 91.5 MB per product on pf 8p+8n at M = 1024,
# position 19, with the grouped passes on every block wider than 32 states (the headline
# superblock is too large for a multi-pass capture; the excess is the intermediate of the
# two-stage passes, which grows with the product); re-take it when the kernels change
HEFF_TRAFFIC_PER_BYTE = 137.4 / 91.5


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


def cpu_oracle_sample(steps, warmup, budget_s=20.0, M0=None):
    """Times the oracle's H_eff products (FP64 numpy) on the headline workload: the
    superblock at position 1 with the starting state's right blocks at M0 states (building
    them is not timed), a seeded random input, repeated until the budget is spent.
    Returns (TFLOP/s, seconds, products, description)."""
    import numpy as np
    from gen import make_problem, initial_mps
    from oracle.dmrg import OracleDMRG
    w = WORKLOAD
    M0 = CPU_SAMPLE_M0 if M0 is None else M0
    prob = make_problem(w["space"], w["Np"], w["Nn"], w["two_Mz"], seed=w["seed"])
    t_setup = time.perf_counter()
    o = OracleDMRG(prob, initial_mps(prob, M0, w["mps_seed"]))
    sb = o.superblock(1)
    t_setup = time.perf_counter() - t_setup
    fl = _oracle_heff_flops(sb)
    x = np.random.default_rng(1).standard_normal(sb.layout.size)
    for _ in range(max(1, warmup)):
        sb.apply(x)
    n, t = 0, 0.0
    while n < max(1, steps) or t < min(budget_s, 10.0):
        t0 = time.perf_counter()
        sb.apply(x)
        t += time.perf_counter() - t0
        n += 1
        if t > budget_s:
            break
    tf = fl * n / max(t, 1e-12) / 1e12
    desc = ("oracle H_eff products of pf 8p+8n (the headline workload) at position 1, "
            "starting-state right blocks of M0=%d states (built in %.0f s, untimed); "
            "psi of %d elements, %.3g GFLOP per product; %d products in %.2f s, FP64 numpy"
            % (M0, t_setup, sb.layout.size, fl / 1e9, n, t))
    return tf, t, n, desc


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"          # before numpy loads: the oracle on one core
    t0 = time.perf_counter()
    tf, secs, nprod, desc = cpu_oracle_sample(args.steps, args.warmup, budget_s=60.0)
    line = {"impl": "reference", "metric": METRIC, "value": tf, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": nprod, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(nprod, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample": desc,
                       "step": "one oracle H_eff product (a whole two-site step of the oracle "
                               "at this size takes hours)"},
            "cpu_baseline": {"value": tf, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": tf, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_baseline_start(steps, warmup):
    """Starts the oracle sample in a child process pinned to one BLAS thread (one of the
    host's cores, beside the GPU work, which the device timers measure)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_oracle_sample(%d, %d)))" % (ROOT, steps, warmup))
    return subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                            stderr=subprocess.DEVNULL, text=True)


def _cpu_baseline_finish(proc):
    """The child's result as the cpu_baseline object (None if it failed)."""
    try:
        out, _ = proc.communicate(timeout=900)
    except subprocess.TimeoutExpired:
        proc.kill()
        proc.communicate()
        return None
    if proc.returncode != 0 or not out.strip():
        return None
    tf, secs, nprod, desc = json.loads(out.strip().splitlines()[-1])
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
    starting state), two-state targeting on pf 4p+4n at M = 1024 in FP64 (one state vs the
    two lowest, from the same starting state), and the all-pairs mutual information of
    pf 4p+4n at M = 256 with the Fiedler order computed from it."""
    import numpy as np
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
    try:
        # the ordering analysis on the device: pf 4p+4n in its natural order, two sweeps at
        # M = 256, then the all-pairs mutual information from a half sweep and the Fiedler
        # order of that matrix
        prob3 = make_problem("pf", 4, 4, 0, seed=2)
        d = P.DMRG(prob3, precision=P.FP64, dav_tol=1e-8)
        d.build_blocks(initial_mps(prob3, 256, 2002))
        d.sweep(256)
        d.sweep(256)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        I, s_i, steps = d.mutual_information(256)
        t_mi = time.perf_counter() - t0
        d.close()
        order, _ = P.fiedler_order(I)
        iu = np.triu_indices(I.shape[0], 1)
        top = np.argsort(I[iu])[::-1][:5]
        out["mutual_information"] = {
            "workload": "pf 4p+4n seed 2, natural order, two FP64 sweeps at M=256, then the "
                        "half sweep of dmrg_mutual_information at M=256",
            "half_sweep_s": t_mi, "energy": steps[-1]["energy"],
            "I_max": float(I.max()), "s_max": float(s_i.max()),
            "top_pairs": [[int(iu[0][k]), int(iu[1][k]), float(I[iu][k])] for k in top],
            "fiedler_order": [int(x) for x in order]}
    except Exception as exc:
        out["mutual_information"] = {"error": str(exc)}
    return out


PFG_SCHEDULE = [(512, 1), (1024, 2), (2048, 1)]


def run_pfg(P, M_max):
    """The pf+g9/2 workload: 60 m-scheme sites, 12p+12n (m-scheme dimension 3.45e14),
    random J-coupled two-body ensemble seed 4, for the targets 2M_z = 0 and 2M_z = 4, mixed
    path, seeded starting state (M0 = 512, seed 4004), schedule 512(1) -> 1024(2) ->
    2048(1) capped at M_max.  Per sweep: seconds (CUDA events), H_eff TFLOP/s on the device,
    energy.  The learned preconditioner is trained on the 2M_z = 0 instance (samples
    harvested during its M = 1024 sweeps) and evaluated on the held-out 2M_z = 4 instance:
    after its schedule, one more sweep at the final M with the diagonal preconditioner, and
    the same sweep from the identical state (a second context through the same
    deterministic schedule) with the learned one."""
    import torch
    from gen import make_problem, initial_mps
    sched = [(M, n) for (M, n) in PFG_SCHEDULE if M <= M_max]
    out = {"workload": "pf+g9/2 60 sites, 12p+12n, seed 4, mixed path, schedule %s" %
                       "+".join("%d(%d)" % x for x in sched)}

    def timed_sweep(d, M):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st, e = d.sweep(M)
        e1.record()
        e1.synchronize()
        fl = sum(x["heff_flops"] * x["n_products"] for x in st)
        hs = sum(x["heff_seconds"] for x in st)
        return st, {"M": M, "s": e0.elapsed_time(e1) / 1e3, "energy": e,
                    "products": sum(x["n_products"] for x in st),
                    "heff_tflops": fl / max(hs, 1e-12) / 1e12,
                    "max_step_gflop": max(x["heff_flops"] for x in st) / 1e9}

    inits = {}

    def run_schedule(tmz, harvest):
        prob = make_problem("pfg", 12, 12, tmz, seed=4)
        if tmz not in inits:
            inits[tmz] = initial_mps(prob, sched[0][0], 4004)
        d = P.DMRG(prob, precision=P.MIXED_FP32, dav_tol=1e-8)
        d.build_blocks(inits[tmz])
        sweeps = []
        for (M, n) in sched:
            for _ in range(n):
                if harvest and M == 1024:
                    d.mlp_harvest(True, 2048)
                sweeps.append(timed_sweep(d, M)[1])
                d.mlp_harvest(False)
        return d, sweeps

    theta = None
    for tmz in (0, 4):
        d, sweeps = run_schedule(tmz, harvest=tmz == 0)
        free_b, total_b = torch.cuda.mem_get_info()
        res = {"sweeps": sweeps, "device_mem_gb": round((total_b - free_b) / 1e9, 2)}
        if tmz == 0:
            d.mlp_reset(3)
            t0 = time.perf_counter()
            loss, ns = d.mlp_train(epochs=20, batch=1024, lr=1e-3, seed=4)
            res["mlp"] = {"samples": ns, "loss": loss, "train_s": time.perf_counter() - t0}
            theta = d.mlp_params()
        elif theta is not None:
            M = sweeps[-1]["M"]
            st_d, sw_d = timed_sweep(d, M)
            d.close()
            d, _ = run_schedule(tmz, harvest=False)     # the identical state again
            d.mlp_set_params(theta)
            d.set_options(precision=P.MIXED_FP32, precond=P.PRECOND_MLP)
            st_l, sw_l = timed_sweep(d, M)
            res["precond_held_out"] = {
                "protocol": "one sweep at M=%d from the identical state, diagonal vs learned "
                            "(network trained on the 2M_z=0 instance)" % M,
                "products_diagonal": sw_d["products"], "products_learned": sw_l["products"],
                "sweep_s_diagonal": sw_d["s"], "sweep_s_learned": sw_l["s"],
                "energy_diagonal": sw_d["energy"], "energy_learned": sw_l["energy"],
                "max_step_dE": max(abs(a["energy"] - b["energy"]) for a, b in zip(st_d, st_l)),
                "max_residual_diagonal": max(x["residual"] for x in st_d),
                "max_residual_learned": max(x["residual"] for x in st_l)}
        d.close()
        out["two_Mz_%d" % tmz] = res
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


SCHEDULE = [(512, 2), (1024, 2), (2048, 2), (4096, 4)]


def _timed_window(N, steps, warmup):
    """(setup, warm-up, timed) positions of a left-to-right pass whose timed steps are
    centred on the middle of the chain."""
    start = max(1, min(N - 2 - steps, N // 2 - 1 - steps // 2))
    w0 = max(1, start - warmup)
    warm = [(p, 0) for p in range(w0, start)]
    setup = [(p, 0) for p in range(1, w0)]
    timed = [(p, 0) for p in range(start, min(N - 2, start + steps))]
    return setup, warm, timed


def _emit(tag, obj):
    """A side measurement on a line of its own (the final line carries the headline)."""
    print(json.dumps({"bench_section": tag, **obj}), flush=True)


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
    # the oracle's CPU sample runs in a child process on one host core while the GPU works
    cpu_proc = None
    if not args.no_cpu_baseline and world == 1:
        cpu_proc = _cpu_baseline_start(args.steps, args.warmup)
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
    schedule = list(SCHEDULE)
    if args.workload:
        # another system of the same family (profiling of smaller cases)
        sp, npr, nne, sd = args.workload.split(":")
        w.update(space=sp, Np=int(npr), Nn=int(nne), seed=int(sd), two_Mz=(int(npr) + int(nne)) % 2)
        wname = "%s shell, %dp+%dn, seed %d (profiling case)" % (sp, int(npr), int(nne), int(sd))
    if args.M != WORKLOAD["M"]:
        schedule = [(m, n) for (m, n) in schedule if m < args.M] + [(args.M, schedule[-1][1])]
    if args.sched_sweeps is not None:
        schedule = [(m, min(n, args.sched_sweeps)) for (m, n) in schedule]
    M = schedule[-1][0]
    prob = make_problem(w["space"], w["Np"], w["Nn"], w["two_Mz"], seed=w["seed"])
    init = initial_mps(prob, schedule[0][0], w["mps_seed"])
    N = prob.n_sites
    with ClockSampler(local) as clk:
        # ---- the whole job through the public API from host arrays (e2e): create the
        # context (Hamiltonian copied from host memory), build the blocks from the host
        # starting state, the sweep schedule, energies read back after every sweep
        h2d = sum(int(a.nbytes) for a in (prob.species, prob.two_m, prob.eps, prob.v_idx,
                                          prob.v_val, prob.order))
        h2d += sum(int(np.asarray(a).nbytes) for a in init.flat())
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_job0 = time.perf_counter()
        d = P.DMRG(prob, precision=P.MIXED_FP32, dav_tol=1e-8, dav_max_iter=args.max_iter)
        d.build_blocks(init)
        sweeps = []
        n_job_steps = 0
        for (Ms, ns) in schedule:
            for _ in range(ns):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                st, e = d.sweep(Ms)
                e1.record()
                e1.synchronize()
                n_job_steps += len(st)
                sweeps.append({"M": Ms, "s": e0.elapsed_time(e1) / 1e3, "energy": e,
                               "products": sum(x["n_products"] for x in st),
                               "heff_flops": sum(x["heff_flops"] * x["n_products"] for x in st),
                               "heff_s": sum(x["heff_seconds"] for x in st),
                               "max_step_ms": 1e3 * max(x["seconds"] for x in st)})
        torch.cuda.synchronize()
        t_job = time.perf_counter() - t_job0
        job_flops = sum(x["heff_flops"] for x in sweeps)
        # work split of the product tuned on the middle superblock at the final M
        tuned_edge, tune_ms = d.autotune(N // 2, reps=2)
        # ---- timed two-site steps at the final M, centred on the middle of the chain
        setup, warm, timed = _timed_window(N, args.steps, args.warmup)
        for (p, dr) in setup + warm:
            d.step(p, dr, M)
        torch.cuda.synchronize()
        c0 = d.counters()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(timed) + 1)]
        stats = []
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
    clocks = clk.summary()
    free_b, total_b = torch.cuda.mem_get_info()
    dev_used_gb = (total_b - free_b) / 1e9
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(timed))]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist)
    flops = sum(s["heff_flops"] * s["n_products"] for s in stats)
    heff_s = sum(s["heff_seconds"] for s in stats)
    heff_bytes = sum(s["heff_bytes"] * s["n_products"] for s in stats)
    nprod = sum(s["n_products"] for s in stats)
    value = replica_throughput(world, flops, total_s)
    peak, peak_kind = _peaks()
    achieved = heff_bytes / max(heff_s, 1e-12) / 1e9
    # ---- one FP64 sweep at M from the state the mixed path reached, step by step; at the
    # middle of the chain (the heaviest superblocks) the mixed and the FP64 Davidson solve
    # the identical superblock first (the energy gate), then the FP64 step continues from
    # the FP64 eigenvector (its Davidson then needs one product: the sweep time is, if
    # anything, slightly in FP64's favour)
    fp64 = {}
    if rank == 0:    # side measurements: rank 0 only (replicas repeat the same work)
        try:
            finish = [(p, 0) for p in range(timed[-1][0] + 1, N - 2)] + \
                     [(p, 1) for p in range(N - 3, 0, -1)]
            for (p, dr) in finish:          # complete the mixed sweep the timed steps are in
                d.step(p, dr, M)
            seq = [(p, 0) for p in range(1, N - 2)] + [(p, 1) for p in range(N - 3, 0, -1)]
            q = N // 2
            fs = []
            for _ in range(max(args.fp64_sweeps, 1) if args.fp64_sweeps > 0 else 0):
                d.set_options(precision=P.FP64, dav_tol=1e-8, dav_max_iter=args.max_iter)
                ms, products, e = 0.0, 0, None
                for (p, dr) in seq:
                    if p == q and dr == 0 and not fp64:
                        d.set_options(precision=P.MIXED_FP32, dav_tol=1e-8,
                                      dav_max_iter=args.max_iter)
                        size = d.psi_layout(q)["size"]
                        psi_m = torch.empty(size, dtype=torch.float64, device="cuda")
                        e_mixed, st_m = d.davidson(q, out=psi_m, allow_noconv=True)
                        d.set_options(precision=P.FP64, dav_tol=1e-8, dav_max_iter=args.max_iter)
                        c2 = d.counters()
                        e_fp64, st_d = d.davidson(q, guess=psi_m, allow_noconv=True)
                        c3 = d.counters()
                        fp64 = {"position": q, "energy": e_fp64, "energy_mixed": e_mixed,
                                "dE_mixed_vs_fp64": abs(e_mixed - e_fp64),
                                "products_mixed": st_m["n_products"],
                                "products_fp64_from_mixed_vector": st_d["n_products"],
                                "converged": [st_m["converged"], st_d["converged"]],
                                "heff_tflops": (c3["heff_flops"] - c2["heff_flops"])
                                / max(c3["heff_seconds"] - c2["heff_seconds"], 1e-12) / 1e12}
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    st = d.step(p, dr, M)
                    e1.record()
                    e1.synchronize()
                    ms += e0.elapsed_time(e1)
                    products += st["n_products"]
                    e = st["energy"]
                fs.append({"s": ms / 1e3, "energy": e, "products": products})
            if fs:
                fp64["sweep_s"] = statistics.median(x["s"] for x in fs)
                fp64["sweeps"] = fs
        except Exception as exc:        # a side measurement never takes the bench line down
            fp64 = {"error": str(exc)}
    d.close()
    del d
    at_M = [x["s"] for x in sweeps if x["M"] == M]
    sweep_s = statistics.median(at_M) if at_M else None
    if rank == 0:
        _emit("schedule", {"workload": wname, "sweeps": sweeps})
        _emit("steps", {"positions": timed, "step_ms": step_ms,
                        "energies": [s["energy"] for s in stats],
                        "products": [s["n_products"] for s in stats],
                        "heff_gflop": [s["heff_flops"] / 1e9 for s in stats],
                        "phase_s": {k: c1[k] - c0[k] for k in ("t_enlarge", "t_super",
                                                                "t_davidson", "t_truncate",
                                                                "t_project", "t_predict",
                                                                "t_sync")},
                        "host_detail_s": [b - a for a, b in zip(c0["t_detail"], c1["t_detail"])],
                        "superblock": {k: c1[k] for k in ("sb_blocks_l", "sb_blocks_r",
                                                           "sb_terms", "sb_tiles",
                                                           "sb_small_tiles", "sb_term_hist")}})
        _emit("fp64", fp64)
    if rank == 0 and args.batch_mcap > 0:
        _emit("batch", run_batch_compare(P, args.batch_mcap))
    if rank == 0 and args.precond:
        _emit("precond", run_precond_compare(P))
    if rank == 0 and args.next_rows:
        _emit("next_rows", run_next_rows(P, prob, init, M, None))
    if rank == 0 and args.pfg_mmax > 0:
        try:
            pfg = run_pfg(P, args.pfg_mmax)
        except Exception as exc:      # a side measurement never takes the bench line down
            pfg = {"error": str(exc)}
        _emit("pfg", pfg)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = _cpu_baseline_finish(cpu_proc) if cpu_proc is not None else None
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": len(timed), "warmup": len(warm), "ms_per_step": 1e3 * total_s / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wname, "M": M,
                   "positions": "%d..%d left to right" % (timed[0][0], timed[-1][0]),
                   "schedule": "+".join("%d(%d)" % x for x in schedule),
                   "autotune": {"heff_big_edge": tuned_edge,
                                "ms_by_edge": {str(k): round(v, 3) for k, v in tune_ms.items()}},
                   "precision": "FP32 contractions (split-TF32 tensor cores), FP64 "
                                "Davidson/SVD/energy",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2: %.0f MB of operator blocks per H_eff product"
                         % (heff_bytes / max(nprod, 1) / 1e6)},
        "heff": {"tflops_device": flops / max(heff_s, 1e-12) / 1e12, "products": nprod,
                 "gflop_per_product": flops / max(nprod, 1) / 1e9,
                 "share_of_steps": heff_s / max(total_s, 1e-12)},
        "sweep_s": {"mixed_median_at_M": sweep_s, "fp64_at_M": fp64.get("sweep_s"),
                    "mixed_energy": sweeps[-1]["energy"] if sweeps else None,
                    "fp64_energy": fp64["sweeps"][-1]["energy"] if fp64.get("sweeps") else None},
        "fp64": {k: fp64.get(k) for k in ("heff_tflops", "dE_mixed_vs_fp64", "position")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": HEFF_TRAFFIC_PER_BYTE * heff_bytes / max(nprod, 1),
                     "kernel": "mixed H_eff product (its kernels between CUDA events on the "
                               "context stream)", "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": {"value": job_flops / t_job / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": h2d / max(n_job_steps, 1),
                "d2h_bytes_per_step": ctypes.sizeof(P.StepStats) + 8,
                "job": "create from host arrays + block build + the schedule (%d sweeps, %d "
                       "steps) with every sweep's step records and energy read back; wall "
                       "clock %.1f s; h2d %d bytes per job" % (len(sweeps), n_job_steps,
                                                               t_job, h2d)},
        "gpu_launches": int(c1["launches"] - c0["launches"]),
        "device_mem_used_gb": round(dev_used_gb, 2),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A small case of the product's kernels for multi-pass ncu captures: pf 8p+8n (seed 3,
    mixed path), sweeps of the schedule up to --M, steps 1..18 left to right at --M, the
    grouped passes on every block wider than --profile-edge states, then inside the profiler
    range either one H_eff product at position 19 ('product') or the two-site step there
    ('step').  Prints one JSON line describing the case."""
    import numpy as np
    import torch
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    from gen import make_problem, initial_mps
    w = WORKLOAD
    M = args.M
    prob = make_problem(w["space"], w["Np"], w["Nn"], w["two_Mz"], seed=w["seed"])
    d = P.DMRG(prob, precision=P.MIXED_FP32)
    d.build_blocks(initial_mps(prob, SCHEDULE[0][0], w["mps_seed"]))
    for m, _ in SCHEDULE:
        if m > M:
            break
        d.sweep(m)
    p = 19
    for q in range(1, p):
        d.step(q, 0, M)
    d.set_tuning(heff_big_edge=args.profile_edge)
    n = d.psi_layout(p)["size"]
    flops, nbytes, _ = d.heff_cost(p)
    x = torch.tensor(np.random.default_rng(1).standard_normal(n), dtype=torch.float64,
                     device="cuda")
    y = torch.empty_like(x)
    d.heff_apply(p, x, y)
    torch.cuda.synchronize()
    free_b, total_b = torch.cuda.mem_get_info()
    torch.cuda.profiler.start()
    out = {"profile_case": args.profile_case, "M": M, "position": p, "psi_size": n,
           "heff_gflop": flops / 1e9, "heff_mb": nbytes / 1e6,
           "device_mem_gb": round((total_b - free_b) / 1e9, 2)}
    if args.profile_case == "product":
        d.heff_apply(p, x, y)
    else:
        st = d.step(p, 0, M)
        out.update(n_products=st["n_products"], kept=st["kept"])
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    d.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--M", type=int, default=WORKLOAD["M"])
    ap.add_argument("--max-iter", type=int, default=100)
    ap.add_argument("--sched-sweeps", type=int, default=None,
                    help="cap the sweeps per M of the schedule (profiling)")
    ap.add_argument("--fp64-sweeps", type=int, default=1,
                    help="FP64 sweeps at the final M after the mixed schedule (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-mcap", type=int, default=2048,
                    help="M cap of the 32-instance batch-vs-loop comparison (0: skip)")
    ap.add_argument("--precond", type=int, default=1,
                    help="learned vs diagonal preconditioner comparison (0: skip)")
    ap.add_argument("--next-rows", type=int, default=1,
                    help="also time a DBSS sweep and a two-state sweep (side measurements)")
    ap.add_argument("--pfg-mmax", type=int, default=2048,
                    help="largest M of the pf+g9/2 12p+12n side measurement (0: skip)")
    ap.add_argument("--workload", default="",
                    help="space:Np:Nn:seed of another system (profiling of smaller cases)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--profile-case", choices=["product", "step"], default=None,
                    help="run only the small capture case at --M (see run_profile_case)")
    ap.add_argument("--profile-edge", type=int, default=32,
                    help="grouped-pass edge of the capture case")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
