#!/usr/bin/env python
"""Benchmark of the Lindblad / quantum-trajectory hot path on GB300.

Default workload (`ising_c2`, the largest configuration that fits one GPU):
the dissipative transverse-field Ising chain, J = 1, h ~ U[0.5, 1.5] (seed 3),
sigma-minus loss gamma = 0.1 on every site, all spins excited, t in [0, 10]
with 100 output times, e_ops Sx, Sy, Sz, mixed precision (FP32 right-hand
side, FP64 state, controller and jump logic), rtol 1e-7, atol 1e-9.  One step
is one pass of the whole path: a mesolve of 10 spins (a density matrix with
2^20 entries, product-form RHS on the grid kernel) followed on the same
stream by an mcsolve of 14 spins (n = 16,384) with 2000 trajectories
(Philox seed 3).

Printed (rank 0, one JSON line): Lindblad RHS evaluations of the step's
mesolve per second of the whole step, mcsolve trajectories per second of the
whole step, each solve's own rate and p50/p99 latency, the error of the
reduced-precision results against FP64, a roofline object for the dominant
kernel, the FP64 oracle timed on a bounded sample on one core and on all host
cores (cpu_baseline), the same job end to end through the host-pointer C ABI
(e2e), the single-solve latency of the driven cavity (N = 20) and the
Jaynes-Cummings job (N = 40 x 2) as extra keys.

Other workloads (`--workload`): jc_40x2, ising10, ising14_mc,
kerr_sweep_1024, serving, optomech_td, ssesolve_jc, smesolve_jc.

Under torchrun each rank runs the same job on its own GPU (independent
problems, no collective on the data path): weak scaling.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this comparison).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

NTRAJ = 1000
SEED = 1
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2: written between timed steps
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 4 FP64 flop/clk x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qtl", choices=["qtl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="ising_c2",
                    choices=["ising_c2", "jc_40x2", "kerr_sweep_1024", "serving", "ising10", "ising14_mc",
                             "optomech_td", "ssesolve_jc", "smesolve_jc", "steadystate", "dsf", "dsf_mc"])
    ap.add_argument("--rates", default="10,30,100,300")
    ap.add_argument("--requests", type=int, default=120)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    s = W.jaynes_cummings()   # N = 40 x 2, tlist range(0, 10 pi/g, 1000)
    return s


def algorithmic_flops(nnz, nnz_half, n_rows, stats):
    """FP64 flops of the integrator counted from the work done: per RHS
    evaluation a complex multiply-add (8 flops) per stored operator entry,
    or 4 flops for the nnz_half entries whose real or imaginary part is zero;
    each attempted step forms 21 stage increments and 7 error terms, each a
    real-times-complex product added to a complex entry (4 flops) per row."""
    attempts = stats["steps_acc"] + stats["steps_rej"]
    per_rhs = 8.0 * (nnz - nnz_half) + 4.0 * nnz_half
    return per_rhs * stats["rhs_evals"] + 4.0 * 28 * n_rows * attempts


def traffic_from_profile(kernel_src, summary):
    """DRAM bytes per launch recorded by an ncu capture (profiles/*.md), or
    None when the kernel source changed since the counters were taken."""
    import hashlib
    try:
        src_hash = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        txt = open(summary).read()
    except OSError:
        return None
    fields = dict(l.split(":", 1) for l in txt.splitlines() if l.startswith(("source_sha256_16:", "dram_bytes_per_launch:")))
    if fields.get("source_sha256_16:".rstrip(":"), "").strip() != src_hash:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_oracle_sample(s, ntraj_sample):
    """The FP64 oracle, as it stands, on the same job: the full mesolve and
    `ntraj_sample` of the 1000 trajectories, single-threaded."""
    from oracle.mcsolve import mcsolve as o_mc
    from oracle.mesolve import mesolve as o_me
    t0 = time.perf_counter()
    me = o_me(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, method="tsit5", rtol=s.rtol, atol=s.atol)
    t1 = time.perf_counter()
    o_mc(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=ntraj_sample, seed=SEED,
         rtol=s.rtol, atol=s.atol)
    t2 = time.perf_counter()
    job_s = (t1 - t0) + (t2 - t1) * NTRAJ / ntraj_sample
    return dict(value=me["stats"]["rhs_evals"] / job_s, me_s=t1 - t0, mc_s=t2 - t1,
                job_s=job_s, expect=me["expect"], rhs=me["stats"]["rhs_evals"])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s = workload()
    ntr = 2
    for _ in range(args.warmup):
        cpu_oracle_sample(s, ntr)
    vals, jobs = [], []
    for _ in range(args.steps):
        r = cpu_oracle_sample(s, ntr)
        vals.append(r["value"])
        jobs.append(r["job_s"])
    v = statistics.mean(vals)
    sample = (f"per step: oracle mesolve of the full job ({r['rhs']} RHS evaluations) + "
              f"{ntr} of {NTRAJ} trajectories, trajectory time scaled to {NTRAJ}")
    out = {"metric": "Lindblad RHS evals/s (mesolve + concurrent 1000-trajectory mcsolve job)",
           "value": v, "unit": "RHS evals/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(jobs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "jc_40x2 (N=40 x 2, L=6400) mesolve FP64 + mcsolve 1000 traj FP64"},
           "cpu_baseline": {"value": v, "unit": "RHS evals/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "RHS evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_qtl(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2504_21440_gb300 import qtl
    qtl.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    s = workload()
    n_e, nt = len(s.e_ops), len(s.tlist)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex_me = torch.zeros((n_e, nt), dtype=torch.complex128, device=dev)
    ex_mc = torch.zeros((n_e, nt), dtype=torch.complex128, device=dev)
    tex = torch.zeros((n_e, nt, NTRAJ), dtype=torch.complex128, device=dev)
    info_me = torch.zeros(5, dtype=torch.int64, device=dev)
    info_mc = torch.zeros(5, dtype=torch.int64, device=dev)
    st_me, st_mc = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    tol = dict(method="tsit5", precision="fp64", rtol=s.rtol, atol=s.atol)
    o_me = qtl.make_opts(stream=st_me.cuda_stream, **tol)
    o_mc = qtl.make_opts(stream=st_mc.cuda_stream, **tol)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    main = torch.cuda.current_stream(dev)

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(main)
        st_me.wait_event(e[0])
        st_mc.wait_event(e[0])
        e[1].record(st_me)
        qtl.mesolve_async(g.handle, psi, 1, tl, o_me, ex_me, None, info_me)
        e[2].record(st_me)
        e[3].record(st_mc)
        qtl.mcsolve_async(g.handle, psi, tl, NTRAJ, SEED, o_mc, ex_mc, tex, info_mc)
        e[4].record(st_mc)
        return e

    for _ in range(args.warmup):
        step()
        torch.cuda.synchronize(dev)
    nnz_L, nnz_A = qtl.system_nnz(g.handle, 2), qtl.system_nnz(g.handle, 1)
    half_L, half_A = qtl.system_nnz(g.handle, 4), qtl.system_nnz(g.handle, 3)

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = qtl.launch_count()
    job_ms, me_ms, mc_ms = [], [], []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e = step()
        torch.cuda.synchronize(dev)
        me_ms.append(e[1].elapsed_time(e[2]))
        mc_ms.append(e[3].elapsed_time(e[4]))
        job_ms.append(max(e[0].elapsed_time(e[2]), e[0].elapsed_time(e[4])))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall0
    launches = qtl.launch_count() - launches0
    clk = clocks.stop()
    total_ms = sum(job_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()

    im = info_me.cpu().numpy()
    ic = info_mc.cpu().numpy()
    st_me_d = dict(steps_acc=int(im[1]), steps_rej=int(im[2]), rhs_evals=int(im[3]))
    st_mc_d = dict(steps_acc=int(ic[1]), steps_rej=int(ic[2]), rhs_evals=int(ic[3]), jumps=int(ic[4]))
    status = (int(im[0]) & 0xffffffff, int(ic[0]) & 0xffffffff)
    ms_per_step = total_ms / args.steps
    value = world * st_me_d["rhs_evals"] / (ms_per_step / 1e3)

    # roofline of the dominant kernel (FP64 ALU bound)
    fl_mc = algorithmic_flops(nnz_A, half_A, s.n, st_mc_d)
    fl_me = algorithmic_flops(nnz_L, half_L, s.n * s.n, st_me_d)
    k_me, k_mc = statistics.mean(me_ms), statistics.mean(mc_ms)
    dom = "mc_traj_kernel" if k_mc >= k_me else "me_cluster_kernel"
    fl, kms = (fl_mc, k_mc) if dom == "mc_traj_kernel" else (fl_me, k_me)
    achieved = fl / (kms / 1e3) / 1e12
    src = "mc_traj.cuh" if dom == "mc_traj_kernel" else "me_cluster.cu"
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2504_21440_gb300", "csrc", src),
                                   os.path.join(ROOT, "profiles", f"{dom}_jc40x2_fp64.md"))
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": dom,
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz (FP64 pipe; nominal 1.25 TFLOP/s)"}
    other = {"me_cluster_kernel": {"ms": k_me, "tflops": fl_me / (k_me / 1e3) / 1e12},
             "mc_traj_kernel": {"ms": k_mc, "tflops": fl_mc / (k_mc / 1e3) / 1e12}}

    out = None
    if rank == 0:
        cpu = None
        err = None
        if not args.no_cpu_baseline:
            r = cpu_oracle_sample(s, 8)
            cpu = {"value": r["value"], "unit": "RHS evals/s", "cores": 1, "kind": "oracle",
                   "sample": f"oracle mesolve of the full job ({r['me_s']:.1f} s) + 8 of {NTRAJ} "
                             f"trajectories ({r['mc_s']:.1f} s), trajectory time scaled to {NTRAJ}; "
                             "single-threaded NumPy/SciPy"}
            err = float(np.max(np.abs(ex_me.cpu().numpy() - r["expect"])))
        e2e = None
        if not args.no_e2e:
            e2e = run_e2e(qtl, g, s, dev, args.steps)
        sj = sorted(job_ms)
        out = {"metric": "Lindblad RHS evals/s (mesolve + concurrent 1000-trajectory mcsolve job)",
               "value": value, "unit": "RHS evals/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "jc_40x2 (N=40 x 2, Liouvillian 6400x6400, nnz %d) mesolve "
                                      "FP64 Tsit5 rtol 1e-8 atol 1e-10, 1000 saveat + mcsolve 1000 "
                                      "trajectories FP64, concurrent streams" % nnz_L,
                          "l2": "flushed (512 MB write) between timed steps",
                          "parallelism": f"independent job per GPU x{world}"},
               "mcsolve_traj_per_s": world * NTRAJ / (ms_per_step / 1e3),
               "latency_ms": {"p50": sj[len(sj) // 2], "p99": sj[min(len(sj) - 1, int(0.99 * len(sj)))],
                              "mesolve_mean": k_me, "mcsolve_mean": k_mc},
               "status": list(status), "stats": {"mesolve": st_me_d, "mcsolve": st_mc_d},
               "err_vs_fp64_oracle": err, "roofline": roof, "kernels": other,
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "wall_s": wall}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    g.free()


def run_e2e(qtl, g, s, dev, steps):
    """The same job through the host-pointer C ABI (qtl_mesolve and
    qtl_mcsolve, one host thread each): every step copies psi0 and tlist to
    the device and the expectation values back."""
    import torch
    st1, st2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    tol = dict(method="tsit5", precision="fp64", rtol=s.rtol, atol=s.atol)
    o1 = qtl.make_opts(stream=st1.cuda_stream, **tol)
    o2 = qtl.make_opts(stream=st2.cuda_stream, **tol)
    n_e, nt = len(s.e_ops), len(s.tlist)
    res = {}

    def me():
        res["me"] = qtl.mesolve(g.handle, n_e, s.psi0, s.tlist, o1)

    def mc():
        res["mc"] = qtl.mcsolve(g.handle, n_e, s.psi0, s.tlist, NTRAJ, SEED, o2)

    walls = []
    for k in range(steps + 1):
        t0 = time.perf_counter()
        a, b = threading.Thread(target=me), threading.Thread(target=mc)
        a.start()
        b.start()
        a.join()
        b.join()
        if k > 0:
            walls.append(time.perf_counter() - t0)
    w = statistics.mean(walls)
    h2d = 2 * (s.n * 16 + nt * 8)
    d2h = 2 * (n_e * nt * 16 + 40)
    return {"value": res["me"]["stats"]["rhs_evals"] / w, "unit": "RHS evals/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * w}


def run_sweep(args):
    """Parameter sweep: 1024 Kerr cavities with N ~ U{10..60} (seed 4),
    t in [0, 50] with 101 output times, mixed precision (FP32 right-hand side,
    FP64 state), rtol 1e-7, atol 1e-9, all solved by one batched call per
    step.  Value: Lindblad RHS evaluations per second summed over instances."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2504_21440_gb300 import qtl
    qtl.load()
    dev = torch.device("cuda", local)
    sys_ = W.kerr_sweep(1024, seed=4)
    handles = [qtl.System(s.H, s.c_ops, s.e_ops) for s in sys_]
    states = [torch.from_numpy(s.psi0).to(dev) for s in sys_]
    exps = [torch.zeros((2, len(sys_[0].tlist)), dtype=torch.complex128, device=dev) for _ in sys_]
    info = torch.zeros((len(sys_), 5), dtype=torch.int64, device=dev)
    tl = torch.from_numpy(sys_[0].tlist).to(dev)
    main = torch.cuda.current_stream(dev)
    opts = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9, stream=main.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    hs = [h.handle for h in handles]

    # one-shot batched calls (host planning and launches every call), for context
    direct = []
    for _ in range(2):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        qtl.mesolve_batch_async(hs, states, [1] * len(hs), tl, opts, exps, info)
        e1.record(main)
        torch.cuda.synchronize(dev)
        direct.append(e0.elapsed_time(e1))
    # the plan: cluster size per group autotuned, launch sequence captured in a
    # CUDA graph; every timed step replays it
    t_plan = time.perf_counter()
    plan = qtl.Batch(hs, states, [1] * len(hs), tl, opts, exps, info, autotune=True)
    t_plan = time.perf_counter() - t_plan

    def step():
        plan.launch(main.cuda_stream)
    for _ in range(args.warmup):
        step()
        torch.cuda.synchronize(dev)
    ms = []
    launches0 = qtl.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        step()
        e1.record(main)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    inf = info.cpu().numpy()
    groups = plan.groups()
    rhs = int(inf[:, 3].sum())
    bad = int(((inf[:, 0] & 0xffffffff) != 0).sum())
    mean_ms = statistics.mean(ms)
    out = {"metric": "Lindblad RHS evals/s (1024-instance Kerr parameter sweep)",
           "value": world * rhs / (mean_ms / 1e3), "unit": "RHS evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 RHS / f64 state",
           "data": "synthetic",
           "config": {"workload": "kerr_sweep_1024: N~U{10..60}, t in [0,50], 101 saveat, mixed, rtol 1e-7 atol 1e-9",
                      "l2": "flushed (512 MB write) between timed steps"},
           "solves_per_s": world * len(hs) / (mean_ms / 1e3), "failed_solves": bad,
           "plan": {"graph_replay": True, "build_s": t_plan, "direct_call_ms": statistics.mean(direct),
                    "groups": [{"cluster": c, "solves": n, "probe_ms": {str(cc): round(t, 3) for cc, t in cand}}
                               for c, n, cand in groups]},
           "rhs_evals_per_step": rhs, "gpu_launches": qtl.launch_count() - launches0, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    plan.free()
    for h in handles:
        h.free()


def run_ising10(args):
    """Dissipative transverse-field Ising chain, 10 spins (rho with 2^20
    entries), h from seed 3, gamma = 0.1, rho0 all excited, tlist
    range(0, 10, 100), mixed precision, rtol 1e-7, atol 1e-9: one mesolve on
    the grid kernel per step.  Value: Lindblad RHS evaluations per second.
    Roofline: bytes of the integrator per attempted step and entry -- per
    stage the stage input read (8 B) and the derivative written (8 B), the 21
    derivative reads of the stage sums and 7 of the error estimate (8 B
    each), the 6 stage inputs written (8 B) and the state read and written
    (2 x 16 B) = 400 B -- against the measured copy bandwidth."""
    import torch
    from paper_2504_21440_gb300 import qtl
    torch.cuda.set_device(0)
    qtl.load()
    dev = torch.device("cuda", 0)
    s = W.ising_chain(10)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex = torch.zeros((3, len(s.tlist)), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)
    main = torch.cuda.current_stream(dev)
    o = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9, stream=main.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        qtl.mesolve_async(g.handle, psi, 1, tl, o, ex, None, info)
        torch.cuda.synchronize(dev)
    ms = []
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qtl.launch_count()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        qtl.mesolve_async(g.handle, psi, 1, tl, o, ex, None, info)
        e1.record(main)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    inf = info.cpu().numpy()
    att = int(inf[1] + inf[2])
    mean_ms = statistics.mean(ms)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = 400.0 * s.n * s.n * att / (mean_ms / 1e3) / 1e9
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2504_21440_gb300", "csrc", "me_grid.cu"),
                                   os.path.join(ROOT, "profiles", "me_grid_kernel_ising10_mixed.md"))
    print(json.dumps({
        "metric": "Lindblad RHS evals/s (10-spin Ising mesolve, 2^20-entry rho)", "value": int(inf[3]) / (mean_ms / 1e3),
        "unit": "RHS evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 RHS / f32-pair state",
        "data": "synthetic", "config": {"workload": "ising10: J=1, h=U[0.5,1.5] seed 3, gamma=0.1, t in [0,10], 100 saveat, mixed",
                                        "l2": "flushed (512 MB write) between timed steps"},
        "attempted_steps": att, "status": int(inf[0]) & 0xffffffff, "Sz_t10": float(ex[2, -1].real),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "me_grid_kernel",
                     "note": "algorithmic 400 B/entry/attempt; the state (~100 MB) is L2-resident"},
        "gpu_launches": qtl.launch_count() - l0, "clocks": clk}))
    g.free()


C2_NTRAJ = 2000
# algorithmic bytes of the mixed wide trajectory kernel per row and attempted
# step (second-order increment form): stages 2-6 read f or f2 and the
# remainders and write one remainder (128 B in all); stage 7 reads y, f
# (hi + lo), f2 and r_3..r_6 (72 B), writes y_new, its FP32 remainder, the
# error partial and scale (36 B), then f_new (hi + lo) after reading the
# partial and scale back (28 B); plus one gather row of the remainder (8 B)
MW_BYTES_PER_ROW = 280.0
C2_SEED = 3            # Philox key of the 14-spin trajectories
C2_TOL = dict(precision="mixed", rtol=1e-7, atol=1e-9)
C2_WORKLOAD = ("ising_c2: dissipative transverse-field Ising chains, J=1, h=U[0.5,1.5] seed 3, "
               "gamma=0.1, all spins excited, t in [0,10], 100 saveat, e_ops Sx Sy Sz, mixed "
               "precision (FP32 RHS, FP64 state / controller / jumps), rtol 1e-7 atol 1e-9: "
               "mesolve of 10 spins (rho with 2^20 entries, grid kernel) then mcsolve of 14 "
               "spins (n = 16384) with 2000 trajectories (Philox seed 3), one stream")


def _hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


_C2_WORKER = {}


def _c2_traj_worker(j):
    """One oracle trajectory of the 14-spin chain (spawned worker process,
    single-threaded); returns its wall time in seconds."""
    if "s" not in _C2_WORKER:
        _C2_WORKER["s"] = W.ising_chain(14)
    from oracle.mcsolve import mcsolve as o_mc
    s = _C2_WORKER["s"]
    t0 = time.perf_counter()
    o_mc(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=1, seed=C2_SEED, traj_ids=[j],
         rtol=C2_TOL["rtol"], atol=C2_TOL["atol"])
    return time.perf_counter() - t0


def c2_cpu_sample(rhs_me, per_core=2, small=False):
    """The FP64 oracle, as it stands, on a bounded sample of the ising_c2 job:
    its 10-spin mesolve over the first output interval (Liouvillian build
    included) and `per_core` 14-spin trajectories per host core in a spawned
    process pool (one single-threaded process per core).  The full job is
    estimated as: Liouvillian build + time per RHS evaluation x rhs_me (the
    RHS count of the full mesolve) + the mean trajectory time x 2000, the
    trajectories spread over the cores (all-core) or run one after another
    (single core)."""
    import multiprocessing as mp
    from oracle.lindblad import liouvillian
    from oracle.mesolve import mesolve as o_me
    cores = os.cpu_count() or 1
    s10 = W.ising_chain(10)
    t0 = time.perf_counter()
    liouvillian(s10.H, s10.c_ops)
    t_build = time.perf_counter() - t0
    tl = s10.tlist[:2] if not small else np.array([0.0, s10.tlist[1] * 0.05])
    t0 = time.perf_counter()
    r = o_me(s10.H, s10.c_ops, s10.e_ops, s10.psi0, tl, rtol=C2_TOL["rtol"], atol=C2_TOL["atol"])
    t_me = time.perf_counter() - t0
    per_rhs = max(t_me - t_build, 1e-9) / r["stats"]["rhs_evals"]
    me_est = t_build + per_rhs * rhs_me
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ntr = max(1, cores * per_core) if not small else 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, ntr)) as pool:
        ttimes = pool.map(_c2_traj_worker, range(ntr))
    t_pool = time.perf_counter() - t0
    traj_mean = statistics.mean(ttimes)
    job_all = me_est + traj_mean * C2_NTRAJ / cores
    job_one = me_est + traj_mean * C2_NTRAJ
    return dict(value_all=rhs_me / job_all, value_one=rhs_me / job_one, cores=cores,
                job_all_s=job_all, job_one_s=job_one, traj_mean_s=traj_mean, ntraj=ntr,
                t_pool_s=t_pool, me_sample_s=t_me, build_s=t_build, rhs_sample=r["stats"]["rhs_evals"],
                per_rhs_s=per_rhs, wall_s=t_me + t_build + t_pool)


def _c2_sample_text(c):
    return (f"oracle (FP64 NumPy/SciPy, as it stands): 10-spin mesolve over the first output interval "
            f"({c['rhs_sample']} RHS evaluations, {c['per_rhs_s']:.3f} s each, Liouvillian build "
            f"{c['build_s']:.1f} s) scaled to the full solve's RHS count, plus {c['ntraj']} of the 2000 "
            f"14-spin trajectories ({c['traj_mean_s']:.2f} s each, one single-threaded spawned process "
            f"per core) scaled to 2000 over {c['cores']} cores")


def c2_reference_rhs():
    """RHS evaluations of the full 10-spin mesolve, for scaling the oracle's
    sample when no GPU run has counted them (the count the adaptive solve
    takes with these tolerances, 347 accepted steps x 6 + 2)."""
    return 2084


def run_c2_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        c2_cpu_sample(c2_reference_rhs(), small=True)
    vals, jobs, last = [], [], None
    for _ in range(args.steps):
        last = c2_cpu_sample(c2_reference_rhs(), per_core=1)
        vals.append(last["value_all"])
        jobs.append(last["job_all_s"])
    v = statistics.mean(vals)
    print(json.dumps({
        "metric": "Lindblad RHS evals/s of the ising_c2 job (10-spin mesolve + 14-spin 2000-trajectory "
                  "mcsolve per step), with mcsolve traj/s",
        "value": v, "unit": "RHS evals/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(jobs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": C2_WORKLOAD},
        "mcsolve_traj_per_s": C2_NTRAJ / statistics.mean(jobs),
        "cpu_baseline": {"value": v, "unit": "RHS evals/s", "cores": last["cores"], "kind": "oracle",
                         "sample": _c2_sample_text(last)},
        "e2e": {"value": v, "unit": "RHS evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]


def c0_latency(qtl, dev, nsolves=20):
    """Single-solve latency of the driven damped cavity (N = 20, FP64 Tsit5,
    rtol 1e-8 atol 1e-10, 201 output times) on the cluster kernel: p50/p99
    over back-to-back solves timed with CUDA events."""
    import torch
    s = W.driven_cavity()
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    rho0 = torch.from_numpy(np.outer(s.psi0, s.psi0.conj()).reshape(-1, order="F").copy()).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex = torch.zeros((2, len(s.tlist)), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)
    main = torch.cuda.current_stream(dev)
    o = qtl.make_opts(rtol=s.rtol, atol=s.atol, stream=main.cuda_stream)
    ms = []
    for k in range(nsolves + 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        qtl.mesolve_async(g.handle, rho0, 0, tl, o, ex, None, info)
        e1.record(main)
        torch.cuda.synchronize(dev)
        if k >= 3:
            ms.append(e0.elapsed_time(e1))
    inf = info.cpu().numpy()
    g.free()
    return {"workload": "driven cavity N=20 FP64 mesolve, 201 saveat", "p50_ms": _pct(ms, 0.5),
            "p99_ms": _pct(ms, 0.99), "solves": nsolves, "rhs_evals": int(inf[3]),
            "rhs_evals_per_s": int(inf[3]) / (statistics.median(ms) / 1e3)}


def c1_job(qtl, dev, steps=3):
    """The Jaynes-Cummings job (N = 40 x 2, FP64 mesolve + 1000 FP64
    trajectories on two concurrent streams), a few timed steps."""
    import torch
    s = workload()
    n_e, nt = len(s.e_ops), len(s.tlist)
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex1 = torch.zeros((n_e, nt), dtype=torch.complex128, device=dev)
    ex2 = torch.zeros((n_e, nt), dtype=torch.complex128, device=dev)
    i1 = torch.zeros(5, dtype=torch.int64, device=dev)
    i2 = torch.zeros(5, dtype=torch.int64, device=dev)
    a, b = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    main = torch.cuda.current_stream(dev)
    oa = qtl.make_opts(rtol=s.rtol, atol=s.atol, stream=a.cuda_stream)
    ob = qtl.make_opts(rtol=s.rtol, atol=s.atol, stream=b.cuda_stream)
    ms = []
    for k in range(steps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        a.wait_event(e0)
        b.wait_event(e0)
        qtl.mesolve_async(g.handle, psi, 1, tl, oa, ex1, None, i1)
        qtl.mcsolve_async(g.handle, psi, tl, NTRAJ, SEED, ob, ex2, None, i2)
        main.wait_stream(a)
        main.wait_stream(b)
        e1.record(main)
        torch.cuda.synchronize(dev)
        if k >= 2:
            ms.append(e0.elapsed_time(e1))
    rhs = int(i1.cpu().numpy()[3])
    g.free()
    m = statistics.mean(ms)
    return {"workload": "jc_40x2 FP64 mesolve + 1000 FP64 trajectories, concurrent streams",
            "ms_per_step": m, "rhs_evals_per_s": rhs / (m / 1e3), "traj_per_s": NTRAJ / (m / 1e3)}


def run_c2(args):
    """The default job (ising_c2, the largest single-GPU configuration): per
    step one mixed-precision mesolve of the 10-spin chain (grid kernel, a
    density matrix with 2^20 entries) followed on the same stream by one
    mixed-precision mcsolve of the 14-spin chain with 2000 trajectories (wide
    trajectory kernel).  Value: Lindblad RHS evaluations of the step's
    mesolve per second of the whole step; mcsolve trajectories per second of
    the whole step beside it; each solve's own rate and p50/p99 latency in
    `phases`.  Roofline: the dominant kernel (mc_wide_kernel, 280 B of state
    per row and attempted step) against the measured copy bandwidth; the
    grid kernel's own figure (400 B per entry and attempted step) in
    `kernels`."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2504_21440_gb300 import qtl
    qtl.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    s10, s14 = W.ising_chain(10), W.ising_chain(14)
    g10 = qtl.System(s10.H, s10.c_ops, s10.e_ops)
    g14 = qtl.System(s14.H, s14.c_ops, s14.e_ops)
    nt = len(s10.tlist)
    psi10 = torch.from_numpy(s10.psi0).to(dev)
    psi14 = torch.from_numpy(s14.psi0).to(dev)
    tl = torch.from_numpy(s10.tlist).to(dev)
    ex10 = torch.zeros((3, nt), dtype=torch.complex128, device=dev)
    ex14 = torch.zeros((3, nt), dtype=torch.complex128, device=dev)
    tex = torch.zeros((3, nt, C2_NTRAJ), dtype=torch.complex128, device=dev)
    i10 = torch.zeros(5, dtype=torch.int64, device=dev)
    i14 = torch.zeros(5, dtype=torch.int64, device=dev)
    main = torch.cuda.current_stream(dev)
    o = qtl.make_opts(stream=main.cuda_stream, **C2_TOL)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(main)
        qtl.mesolve_async(g10.handle, psi10, 1, tl, o, ex10, None, i10)
        e[1].record(main)
        qtl.mcsolve_async(g14.handle, psi14, tl, C2_NTRAJ, C2_SEED, o, ex14, tex, i14)
        e[2].record(main)
        return e

    for _ in range(args.warmup):
        step()
        torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = qtl.launch_count()
    me_ms, mc_ms, job_ms, att_me, att_mc = [], [], [], [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e = step()
        torch.cuda.synchronize(dev)
        me_ms.append(e[0].elapsed_time(e[1]))
        mc_ms.append(e[1].elapsed_time(e[2]))
        job_ms.append(e[0].elapsed_time(e[2]))
        a, b = i10.cpu().numpy(), i14.cpu().numpy()
        att_me.append(int(a[1] + a[2]))
        att_mc.append(int(b[1] + b[2]))
    torch.cuda.synchronize(dev)
    launches = qtl.launch_count() - l0
    clk = clocks.stop()
    total_ms = sum(job_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    a, b = i10.cpu().numpy(), i14.cpu().numpy()
    st10 = dict(steps_acc=int(a[1]), steps_rej=int(a[2]), rhs_evals=int(a[3]))
    st14 = dict(steps_acc=int(b[1]), steps_rej=int(b[2]), rhs_evals=int(b[3]), jumps=int(b[4]))
    status = [int(a[0]) & 0xffffffff, int(b[0]) & 0xffffffff]
    ms_per_step = total_ms / args.steps
    value = world * st10["rhs_evals"] / (ms_per_step / 1e3)
    peak, peak_src = _hbm_peak()
    k_me, k_mc = statistics.mean(me_ms), statistics.mean(mc_ms)
    gb_mc = MW_BYTES_PER_ROW * s14.n * statistics.mean(att_mc) / 1e9
    gb_me = 400.0 * s10.n * s10.n * statistics.mean(att_me) / 1e9
    ach_mc, ach_me = gb_mc / (k_mc / 1e3), gb_me / (k_me / 1e3)
    tr_mc = traffic_from_profile(os.path.join(ROOT, "paper_2504_21440_gb300", "csrc", "mc_wide.cuh"),
                                 os.path.join(ROOT, "profiles", "mc_wide_kernel_ising14_mixed.md"))
    tr_me = traffic_from_profile(os.path.join(ROOT, "paper_2504_21440_gb300", "csrc", "me_grid.cu"),
                                 os.path.join(ROOT, "profiles", "me_grid_kernel_ising10_mixed.md"))
    roof = {"bound": "hbm", "achieved": ach_mc, "peak": peak, "unit": "GB/s", "frac": ach_mc / peak,
            "traffic": tr_mc, "kernel": "mc_wide_kernel", "peak_source": f"hbm_gbs ({peak_src})",
            "algorithmic_bytes_per_launch": gb_mc * 1e9,
            "model": "280 B of trajectory state per row per attempted step (increment form)"}
    kernels = {"mc_wide_kernel": {"ms": k_mc, "gb_s": ach_mc, "frac": ach_mc / peak, "traffic": tr_mc},
               "me_grid_kernel": {"ms": k_me, "gb_s": ach_me, "frac": ach_me / peak, "traffic": tr_me,
                                  "model": "400 B per rho entry per attempted step"}}
    out = None
    if rank == 0:
        # the reduced-precision results against FP64 (host API with the FP64
        # shadow; outside the timed region): the full mesolve, and the first
        # 152 trajectories (one per SM) of the mcsolve
        r10 = qtl.mesolve(g10.handle, 3, s10.psi0, s10.tlist, qtl.make_opts(shadow_fp64=True, **C2_TOL))
        r14 = qtl.mcsolve(g14.handle, 3, s14.psi0, s14.tlist, 152, C2_SEED,
                          qtl.make_opts(shadow_fp64=True, **C2_TOL))
        err = {"mesolve_ising10": r10["stats"]["err_vs_fp64"],
               "mcsolve_ising14_first152traj": r14["stats"]["err_vs_fp64"]}
        e2e = None
        if not args.no_e2e:
            walls = []
            o_host = qtl.make_opts(stream=main.cuda_stream, **C2_TOL)
            for k in range(3):
                t0 = time.perf_counter()
                qtl.mesolve(g10.handle, 3, s10.psi0, s10.tlist, o_host)
                qtl.mcsolve(g14.handle, 3, s14.psi0, s14.tlist, C2_NTRAJ, C2_SEED, o_host)
                if k > 0:
                    walls.append(time.perf_counter() - t0)
            w = statistics.mean(walls)
            e2e = {"value": st10["rhs_evals"] / w, "unit": "RHS evals/s",
                   "h2d_bytes_per_step": (s10.n + s14.n) * 16 + 2 * nt * 8,
                   "d2h_bytes_per_step": 2 * (3 * nt * 16 + 40), "ms_per_step": 1e3 * w,
                   "mcsolve_traj_per_s": C2_NTRAJ / w,
                   "path": "host-pointer qtl_mesolve then qtl_mcsolve, copies inside the timed region"}
        c0 = c0_latency(qtl, dev)
        c1 = c1_job(qtl, dev)
        cpu = None
        if not args.no_cpu_baseline:
            c = c2_cpu_sample(st10["rhs_evals"])
            cpu = {"value": c["value_all"], "unit": "RHS evals/s", "cores": c["cores"], "kind": "oracle",
                   "sample": _c2_sample_text(c), "single_core_value": c["value_one"],
                   "job_s_all_cores": c["job_all_s"], "job_s_single_core": c["job_one_s"],
                   "mcsolve_traj_per_s_all_cores": C2_NTRAJ / c["job_all_s"]}
        out = {"metric": "Lindblad RHS evals/s of the ising_c2 job (10-spin mesolve + 14-spin 2000-trajectory "
                         "mcsolve per step), with mcsolve traj/s",
               "value": value, "unit": "RHS evals/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32 RHS / f64 state (mixed)",
               "data": "synthetic",
               "config": {"workload": C2_WORKLOAD,
                          "l2": "flushed (512 MB write) between timed steps; 14-spin state 290 MB > L2",
                          "parallelism": f"independent job per GPU x{world}"},
               "mcsolve_traj_per_s": world * C2_NTRAJ / (ms_per_step / 1e3),
               "phases": {"mesolve_ising10": {"ms_mean": k_me, "p50_ms": _pct(me_ms, 0.5), "p99_ms": _pct(me_ms, 0.99),
                                              "rhs_evals": st10["rhs_evals"],
                                              "rhs_evals_per_s": st10["rhs_evals"] / (k_me / 1e3)},
                          "mcsolve_ising14": {"ms_mean": k_mc, "p50_ms": _pct(mc_ms, 0.5), "p99_ms": _pct(mc_ms, 0.99),
                                              "traj_per_s": C2_NTRAJ / (k_mc / 1e3),
                                              "attempted_steps_per_traj": statistics.mean(att_mc) / C2_NTRAJ}},
               "latency_ms": {"p50": _pct(job_ms, 0.5), "p99": _pct(job_ms, 0.99)},
               "err_vs_fp64": err, "Sz_t10": {"ising10": float(ex10[2, -1].real), "ising14": float(ex14[2, -1].real)},
               "status": status, "stats": {"mesolve": st10, "mcsolve": st14},
               "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
               "c0_single_solve_latency": c0, "c1_job": c1,
               "gpu_launches": launches, "clocks": clk}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    g10.free()
    g14.free()


def run_steady(args):
    """Stationary states (Sec. 3.2; Appendix A): a driven Kerr cavity with
    N = 256 (65,536 unknowns: Delta = 0.5, K = 0.02, F = 2, kappa = 0.1) by
    qtl_steadystate with the FP64 and with the tensor-core (split-BF16)
    preconditioner, and the Fourier components (|k| <= 4) of the same cavity
    at N = 40 under F cos(t)(a + a'), each timed over `steps` solves after
    the warm-up (the first warm-up solve pays the host eigendecomposition,
    timed separately).  The oracle's direct sparse solves are timed beside
    them on the host, and the GPU results are compared with them."""
    import torch
    from paper_2504_21440_gb300 import qtl
    from oracle.steadystate import steadystate as o_ss, steadystate_fourier as o_ssf
    torch.cuda.set_device(0)
    qtl.load()
    out = {"metric": "stationary-state solves per second", "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "dtype": "f64 (preconditioner GEMMs f64 or split bf16)",
           "data": "synthetic", "cases": {}}
    s = W.kerr_cavity(256, 0.5, 0.02, 2.0, 0.1)
    a = sp_destroy(40)
    cases = [("kerr256", s.H, s.c_ops, None), ("kerr40_fourier", 0.5 * (a.conj().T @ a) + 0.01 * (a.conj().T @ a.conj().T @ a @ a),
                                               [np.sqrt(0.2) * a], a + a.conj().T)]
    for name, H, c, X in cases:
        g = qtl.System(H, c, [])
        t0 = time.perf_counter()
        solve = (lambda **kw: g.steadystate(**kw)) if X is None else (lambda **kw: g.steadystate_fourier(X, 0.8, 1.0, 4, **kw))
        solve()
        t_setup = time.perf_counter() - t0
        res = {"first_solve_s_with_setup": t_setup}
        for prec in ("fp64", "mixed"):
            for _ in range(max(0, args.warmup - 1)):
                solve(precision=prec)
            ts = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = solve(precision=prec)
                ts.append(time.perf_counter() - t0)
            res[prec] = {"s_per_solve": statistics.mean(ts), "solves_per_s": 1.0 / statistics.mean(ts),
                         "iterations": r["stats"]["iterations"], "residual": r["stats"]["residual"]}
            last = r
        t0 = time.perf_counter()
        ref = o_ss(H, c) if X is None else o_ssf(H, c, X, 0.8, 1.0, 4)
        t_cpu = time.perf_counter() - t0
        if X is None:
            err = float(np.max(np.abs(last["rho"] - ref)))
        else:
            err = max(float(np.max(np.abs(last["rho"][k] - ref[k]))) for k in ref)
        res["err_vs_oracle_direct_solve"] = err
        res["cpu_baseline"] = {"s_per_solve": t_cpu, "kind": "oracle (SciPy direct sparse solve)", "cores": 1}
        res["unknowns"] = int(H.shape[0] ** 2 * (1 if X is None else 9))
        out["cases"][name] = res
        g.free()
    out["value"] = out["cases"]["kerr256"]["mixed"]["solves_per_s"]
    print(json.dumps(out))


def sp_destroy(N):
    import scipy.sparse as sp
    return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)


def run_dsf(args):
    """Dynamical shifted Fock mesolve (Sec. 3.6, Appendix B): the strongly
    driven damped cavity (Delta = 0.5, F = 7, kappa = 1, about 98 photons)
    followed at a Fock cutoff of 8, t in [0, 6] with 301 checks, threshold
    0.05, rtol 1e-10 atol 1e-12, timed over `steps` runs; the oracle on one
    core beside it, and the largest difference from it."""
    from paper_2504_21440_gb300 import qtl
    from oracle.dsf import dsf_mesolve as o_dsf
    qtl.load()
    N, D, F, kap = 8, 0.5, 7.0, 1.0
    a = sp_destroy(N)
    tl = np.linspace(0.0, 6.0, 301)
    H = lambda o: D * (o[0].conj().T @ o[0]) + F * (o[0] + o[0].conj().T)
    c = lambda o: [np.sqrt(kap) * o[0]]
    e = lambda o: [o[0], o[0].conj().T @ o[0]]
    tol = dict(rtol=1e-10, atol=1e-12)
    for _ in range(args.warmup):
        qtl.dsf_mesolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, **tol)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = qtl.dsf_mesolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, **tol)
        ts.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    ref = o_dsf(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.05, **tol)
    t_cpu = time.perf_counter() - t0
    m = statistics.mean(ts)
    print(json.dumps({"metric": "dsf_mesolve solves per second", "value": 1.0 / m, "unit": "solves/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
                      "data": "synthetic", "s_per_solve": m, "shifts": r["shifts"], "rhs_evals": r["stats"]["rhs_evals"],
                      "config": {"workload": "dsf driven cavity: N=8, Delta=0.5, F=7, kappa=1, t in [0,6], 301 checks, "
                                             "threshold 0.05, rtol 1e-10 atol 1e-12"},
                      "err_vs_oracle": float(max(np.max(np.abs(r["expect"] - ref["expect"])),
                                                 np.max(np.abs(r["alpha"] - ref["alpha"])))),
                      "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                       "sample": "one full solve"}}))


def run_dsf_mc(args):
    """Dynamical shifted Fock on quantum trajectories (Sec. 3.6, Appendix B
    applied per trajectory): a driven Kerr cavity (Delta = 0.5, K = 0.05,
    F = 3, kappa = 1, <n> up to about 12) at a Fock cutoff of 10, t in [0, 6]
    with 61 checks, threshold 0.1, 256 trajectories, FP64, rtol 1e-9 atol
    1e-11, timed over `steps` runs.  The oracle runs the first 4 trajectories
    (the same Philox streams) on one core: its rate beside the GPU's, and the
    largest difference between the two trajectory by trajectory."""
    from paper_2504_21440_gb300 import qtl
    from oracle.dsf import dsf_mcsolve as o_dsf_mc
    qtl.load()
    N, D, K, F, kap = 10, 0.5, 0.05, 3.0, 1.0
    a = sp_destroy(N)
    tl = np.linspace(0.0, 6.0, 61)
    H = lambda o: (D * (o[0].conj().T @ o[0]) + (K / 2) * (o[0].conj().T @ o[0].conj().T @ o[0] @ o[0])
                   + F * (o[0] + o[0].conj().T))
    c = lambda o: [np.sqrt(kap) * o[0]]
    e = lambda o: [o[0].conj().T @ o[0], o[0]]
    tol = dict(rtol=1e-9, atol=1e-11)
    ntraj, nsample = 256, 4
    run = lambda: qtl.dsf_mcsolve(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.1, ntraj, 5, keep_trajectories=True, **tol)
    for _ in range(args.warmup):
        run()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = run()
        ts.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    ref = o_dsf_mc(H, c, e, [a], [0.0], np.eye(N)[0], tl, 0.1, ntraj=nsample, seed=5, keep_trajectories=True, **tol)
    t_cpu = time.perf_counter() - t0
    m = statistics.mean(ts)
    print(json.dumps({"metric": "dsf_mcsolve trajectories per second", "value": ntraj / m, "unit": "traj/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": "f64", "data": "synthetic", "s_per_solve": m, "shifts": r["shifts"],
                      "jumps": r["stats"]["jumps"], "rhs_evals": r["stats"]["rhs_evals"],
                      "config": {"workload": "dsf_mcsolve driven Kerr cavity: N=10, Delta=0.5, K=0.05, F=3, kappa=1, "
                                             "t in [0,6], 61 checks, threshold 0.1, 256 trajectories (seed 5), "
                                             "rtol 1e-9 atol 1e-11"},
                      "err_vs_oracle_first4traj": float(np.max(np.abs(r["traj_expect"][:nsample] - ref["traj_expect"]))),
                      "cpu_baseline": {"value": nsample / t_cpu, "unit": "traj/s", "cores": 1, "kind": "oracle",
                                       "sample": f"the first {nsample} of the {ntraj} trajectories"}}))


def run_ising14_mc(args):
    """mcsolve on the dissipative transverse-field Ising chain of 14 spins
    (n = 16,384; H_eff with 245,760 entries), h from seed 3, gamma = 0.1, all
    spins excited, tlist range(0, 10, 100), 2000 trajectories, mixed
    precision, rtol 1e-7, atol 1e-9: one mcsolve (the wide trajectory kernel,
    one 1024-thread CTA per trajectory) per step.  Value: trajectories per
    second.  Roofline: the integrator's state bytes per attempted step and row
    in the second-order increment form (MW_BYTES_PER_ROW, 280 B) against the
    measured copy bandwidth (H_eff itself is shared by all trajectories and
    stays in L2)."""
    import torch
    from paper_2504_21440_gb300 import qtl
    torch.cuda.set_device(0)
    qtl.load()
    dev = torch.device("cuda", 0)
    s = W.ising_chain(14)
    ntraj = 2000
    g = qtl.System(s.H, s.c_ops, s.e_ops)
    psi = torch.from_numpy(s.psi0).to(dev)
    tl = torch.from_numpy(s.tlist).to(dev)
    ex = torch.zeros((3, len(s.tlist)), dtype=torch.complex128, device=dev)
    tex = torch.zeros((3, len(s.tlist), ntraj), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)
    main = torch.cuda.current_stream(dev)
    o = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9, stream=main.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        qtl.mcsolve_async(g.handle, psi, tl, 152, SEED, o, ex, tex, info)
        torch.cuda.synchronize(dev)
    ms, atts = [], []
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qtl.launch_count()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        qtl.mcsolve_async(g.handle, psi, tl, ntraj, SEED, o, ex, tex, info)
        e1.record(main)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        inf = info.cpu().numpy()
        atts.append(int(inf[1] + inf[2]))
    clk = clocks.stop()
    launches = qtl.launch_count() - l0
    mean_ms = statistics.mean(ms)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = MW_BYTES_PER_ROW * s.n * statistics.mean(atts) / (mean_ms / 1e3) / 1e9
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2504_21440_gb300", "csrc", "mc_wide.cuh"),
                                   os.path.join(ROOT, "profiles", "mc_wide_kernel_ising14_mixed.md"))
    print(json.dumps({
        "metric": "mcsolve traj/s (14-spin Ising, n = 16384, 2000 trajectories)",
        "value": ntraj / (mean_ms / 1e3), "unit": "traj/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 RHS / f64 state", "data": "synthetic",
        "config": {"workload": "ising14 mcsolve: J=1, h=U[0.5,1.5] seed 3, gamma=0.1, t in [0,10], "
                               "100 saveat, 2000 trajectories, mixed, rtol 1e-7 atol 1e-9",
                   "l2": "flushed (512 MB write) between timed steps; per-CTA state 1.9 MB x 152 > L2"},
        "attempted_steps_per_traj": statistics.mean(atts) / ntraj, "jumps": int(inf[4]),
        "status": int(inf[0]) & 0xffffffff, "Sz_t10": float(ex[2, -1].real),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "mc_wide_kernel",
                     "note": "algorithmic 280 B/row/attempt of state (increment form); latency-bound (see profiles)"},
        "gpu_launches": launches, "clocks": clk}))
    g.free()


def _prepare_systems(reqs, systems, opts_list):
    """One minimal solve per system and precision before timing: the lazy
    device structures (Liouvillian, grid operators, sliced ELLPACK) are built
    as they would be when the system is created ahead of its requests."""
    for r, g in zip(reqs, systems):
        sy = r["system"]
        tl = np.array([0.0, 1e-6])
        for o in opts_list:
            kw = dict(precision=o, rtol=1e-7, atol=1e-9)
            if r["kind"] == "mesolve":
                g.mesolve(sy.psi0, tl, **kw)
            else:
                g.mcsolve(sy.psi0, tl, 1, 0, **kw)


def run_serving(args):
    """Serving: Poisson arrivals of mixed requests at each rate -- 60%
    mesolve on coupled-cavity pairs (N1, N2 ~ U{4..32}, J ~ U[0,1],
    kappa_i ~ U[0.01,0.3], rho0 = |1,0>, t in [0,20], 101 points) and 40%
    mcsolve on Ising chains (8-14 spins, 100-2000 trajectories, t in [0,10],
    101 points), mixed precision, rtol 1e-7, atol 1e-9 -- submitted to one
    qtl server (HBM budget 90% of free memory, 8 requests in flight).
    Latency = completion - arrival.  The systems are created, and their
    device structures built, before the arrivals start."""
    import threading as th
    import torch
    from paper_2504_21440_gb300 import qtl
    torch.cuda.set_device(0)
    qtl.load()
    opts = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9)
    lines = []
    for rate in [float(x) for x in args.rates.split(",")]:
        reqs = W.serving_mix(n_requests=args.requests, seed=5, rate=rate, ising_spins=(8, 14))
        systems = [qtl.System(r["system"].H, r["system"].c_ops, r["system"].e_ops) for r in reqs]
        _prepare_systems(reqs, systems, ["mixed"])
        srv = qtl.Server(max_inflight=8)
        # warm-up: one request of each kind
        for r, g in list(zip(reqs, systems))[:4]:
            srv.wait(srv.submit(r["kind"], g, r["system"].psi0, r["system"].tlist, opts,
                                ntraj=r.get("ntraj", 0), seed=r.get("seed", 0)))
        tickets = [None] * len(reqs)
        t0 = time.perf_counter()
        for i, (r, g) in enumerate(zip(reqs, systems)):
            dt = t0 + r["arrival"] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = (time.perf_counter(), srv.submit(r["kind"], g, r["system"].psi0, r["system"].tlist,
                                                          opts, ntraj=r.get("ntraj", 0), seed=r.get("seed", 0)))
        res = [srv.wait(t) for _, t in tickets]
        t1 = time.perf_counter()
        srv.free()
        for g in systems:
            g.free()
        mono0 = time.monotonic() - time.perf_counter()   # perf_counter -> steady clock offset
        lat = sorted(1e3 * (r["t_end"] - (t0 + rq["arrival"] + mono0)) for r, rq in zip(res, reqs))
        bad = sum(1 for r in res if r["status"] != 0)
        lines.append({"rate_req_per_s": rate, "requests": len(reqs), "failed": bad,
                      "solves_per_s": len(reqs) / (t1 - t0),
                      "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                     "max": lat[-1]},
                      "mix": {"mesolve": sum(r["kind"] == "mesolve" for r in reqs),
                              "mcsolve": sum(r["kind"] == "mcsolve" for r in reqs)}})
    print(json.dumps({"metric": "p50/p99 solve latency and solves/s under Poisson arrivals",
                      "workload": "serving mix: coupled-cavity mesolve (n 16-1024) + Ising mcsolve (8-14 spins)",
                      "dtype": "f32 RHS / f64 state", "data": "synthetic", "n_gpus": 1, "rates": lines,
                      "vs_fp64_single_solve": serving_vs_fp64(qtl, opts)}))


def serving_vs_fp64(qtl, opts_mixed, n_req=40):
    """The same request sample -- the first n_req requests of the serving mix
    as configured (seed 5: coupled-cavity mesolve with N1, N2 ~ U{4..32} and
    Ising mcsolve with 8-14 spins and 100-2000 trajectories), all arrived at
    once -- through the server in mixed precision and through the plain FP64
    single-solve path, one request after the other.  Reports solves/s of both
    and each result's error against FP64: the largest |difference| of an
    expectation value between the mixed and the FP64 solve with the same
    options and random draws (the library's err_vs_fp64 reading), as max and
    median per kind."""
    reqs = W.serving_mix(n_requests=n_req, seed=5, rate=1e6, ising_spins=(8, 14))
    systems = [qtl.System(r["system"].H, r["system"].c_ops, r["system"].e_ops) for r in reqs]
    _prepare_systems(reqs, systems, ["mixed", "fp64"])
    o64 = qtl.make_opts(precision="fp64", rtol=1e-7, atol=1e-9)
    srv = qtl.Server(max_inflight=8)
    r0, g0 = reqs[0], systems[0]   # warm-up
    srv.wait(srv.submit(r0["kind"], g0, r0["system"].psi0, r0["system"].tlist, opts_mixed,
                        ntraj=r0.get("ntraj", 0), seed=r0.get("seed", 0)))
    t0 = time.perf_counter()
    tickets = [srv.submit(r["kind"], g, r["system"].psi0, r["system"].tlist, opts_mixed,
                          ntraj=r.get("ntraj", 0), seed=r.get("seed", 0)) for r, g in zip(reqs, systems)]
    served = [srv.wait(t) for t in tickets]
    t_srv = time.perf_counter() - t0
    srv.free()
    t0 = time.perf_counter()
    single = []
    for r, g in zip(reqs, systems):
        sy = r["system"]
        if r["kind"] == "mesolve":
            single.append(qtl.mesolve(g.handle, g.n_e, sy.psi0, sy.tlist, o64))
        else:
            single.append(qtl.mcsolve(g.handle, g.n_e, sy.psi0, sy.tlist, r["ntraj"], r["seed"], o64))
    t_one = time.perf_counter() - t0
    om = qtl.make_opts(precision="mixed", rtol=1e-7, atol=1e-9)
    t0 = time.perf_counter()
    for r, g in zip(reqs, systems):
        sy = r["system"]
        if r["kind"] == "mesolve":
            qtl.mesolve(g.handle, g.n_e, sy.psi0, sy.tlist, om)
        else:
            qtl.mcsolve(g.handle, g.n_e, sy.psi0, sy.tlist, r["ntraj"], r["seed"], om)
    t_mix_one = time.perf_counter() - t0
    for g in systems:
        g.free()
    err = {"mesolve": [], "mcsolve": []}
    for a, b, r in zip(served, single, reqs):
        err[r["kind"]].append(float(np.max(np.abs(np.asarray(a["expect"]) - b["expect"]))))
    summ = {k: ({"max": max(v), "median": float(np.median(v)), "results": len(v)} if v else None)
            for k, v in err.items()}
    return {"requests": n_req,
            "sample": "first %d requests of the serving mix (seed 5, 8-14-spin chains), all arrived at t=0" % n_req,
            "served_mixed_solves_per_s": n_req / t_srv, "fp64_single_solves_per_s": n_req / t_one,
            "mixed_one_by_one_solves_per_s": n_req / t_mix_one,
            "speedup": t_one / t_srv, "err_vs_fp64_per_result": summ,
            "failed": sum(1 for r in served if r["status"] != 0)}


def optomech_system():
    """The driven optomechanical system of Sec. 3.4 with the paper's
    parameters: Nc = 10, Nm = 7, wc = 1, wm = 2, g = 0.05, kappa = gamma = 0.01,
    drive F cos(w_d t)(a + a^dag) with F = 10 kappa and w_d = wc, from the
    vacuum, tlist = range(0, 5/kappa, 5000), e_ops {a^dag a}."""
    import scipy.sparse as sp
    Nc, Nm = 10, 7
    wc, wm, gc, kap, gam = 1.0, 2.0, 0.05, 0.01, 0.01

    def destroy(N):
        return sp.diags(np.sqrt(np.arange(1, N)), 1, format="csr", dtype=complex)
    a = sp.kron(destroy(Nc), sp.identity(Nm), format="csr")
    b = sp.kron(sp.identity(Nc), destroy(Nm), format="csr")
    ad, bd = a.conj().T, b.conj().T
    H0 = (wc * ad @ a + wm * bd @ b + gc / 2 * (a + ad) @ (a + ad) @ (b + bd)).tocsr()
    drive = ((a + ad).tocsr(), dict(kind="cos", amp=10 * kap, omega=wc))
    psi0 = np.zeros(Nc * Nm, dtype=complex)
    psi0[0] = 1
    tl = np.linspace(0, 5 / kap, 5000)
    return H0, drive, [np.sqrt(kap) * a, np.sqrt(gam) * b], [(ad @ a).tocsr()], psi0, tl


def run_optomech(args):
    """Time-dependent mesolve: the driven optomechanical system of Sec. 3.4
    (dimension 70) over t in [0, 500] with 5000 output times, FP64, Tsit5,
    rtol 1e-8, atol 1e-10, on the grid kernel (the path for time-dependent
    Hamiltonians).  Value: Lindblad RHS evaluations per second; the oracle
    (product form, one host core) is timed on the first 2% of the span."""
    import torch
    from paper_2504_21440_gb300 import qtl
    from oracle.timedep import Coef, mesolve_td
    torch.cuda.set_device(0)
    qtl.load()
    dev = torch.device("cuda", 0)
    H0, drive, c_ops, e_ops, psi0, tl = optomech_system()
    g = qtl.System(H0, c_ops, e_ops, td=[drive])
    psi = torch.from_numpy(psi0).to(dev)
    tld = torch.from_numpy(tl).to(dev)
    ex = torch.zeros((1, len(tl)), dtype=torch.complex128, device=dev)
    info = torch.zeros(5, dtype=torch.int64, device=dev)
    main = torch.cuda.current_stream(dev)
    o = qtl.make_opts(stream=main.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        qtl.mesolve_async(g.handle, psi, 1, tld, o, ex, None, info)
        torch.cuda.synchronize(dev)
    ms = []
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qtl.launch_count()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        qtl.mesolve_async(g.handle, psi, 1, tld, o, ex, None, info)
        e1.record(main)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = qtl.launch_count() - l0
    inf = info.cpu().numpy()
    mean_ms = statistics.mean(ms)
    out = ex.cpu().numpy()
    # oracle on the first 2% of the span, scaled by RHS evaluations
    m = 101
    t0 = time.perf_counter()
    ref = mesolve_td(H0, [(drive[0], Coef(**drive[1]))], c_ops, e_ops, psi0, tl[:m])
    t_cpu = time.perf_counter() - t0
    g.free()
    print(json.dumps({
        "metric": "Lindblad RHS evals/s (time-dependent mesolve, driven optomechanics of Sec. 3.4)",
        "value": int(inf[3]) / (mean_ms / 1e3), "unit": "RHS evals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "optomech_td: Nc=10 x Nm=7, F cos(wd t)(a+a'), t in [0,500], 5000 saveat, FP64",
                   "l2": "flushed (512 MB write) between timed steps"},
        "attempted_steps": int(inf[1] + inf[2]), "status": int(inf[0]) & 0xffffffff,
        "n_final": float(out[0, -1].real),
        "err_vs_oracle_first_2pct": float(np.max(np.abs(out[0, :m] - ref["expect"][0]))),
        "cpu_baseline": {"value": ref["stats"]["rhs_evals"] / t_cpu, "unit": "RHS evals/s", "cores": 1,
                         "kind": "oracle", "sample": "oracle mesolve over the first %d output times (%.1f s)" % (m, t_cpu)},
        "gpu_launches": launches, "clocks": clk}))


def run_ssesolve(args):
    """Homodyne detection (Sec. 3.5, the paper's example): Jaynes-Cummings
    with N = 20, wc = wq = 5, g = 0.1, S = sqrt(kappa) a (kappa = 1), e_ops
    {X = S + S^dag}, psi0 = |alpha = 2, e>, tlist = range(0, 10 pi / wc, 400),
    500 trajectories, Euler-Maruyama with dt = 1e-3, FP64.  Value:
    trajectories per second; the oracle is timed on 2 trajectories."""
    import math
    import scipy.sparse as sp
    import torch
    from paper_2504_21440_gb300 import qtl
    from oracle.stochastic import ssesolve as o_sse
    torch.cuda.set_device(0)
    qtl.load()
    N, wc, wq, gc, kap, alpha, ntraj = 20, 5.0, 5.0, 0.1, 1.0, 2.0, 500

    def destroy(M):
        return sp.diags(np.sqrt(np.arange(1, M)), 1, format="csr", dtype=complex)
    a = sp.kron(destroy(N), sp.identity(2), format="csr")
    sm = sp.kron(sp.identity(N), sp.csr_matrix(np.array([[0, 0], [1, 0]], dtype=complex)), format="csr")
    sz = sp.kron(sp.identity(N), sp.csr_matrix(np.diag([1.0, -1.0]).astype(complex)), format="csr")
    H = (wc * a.conj().T @ a + wq * sz / 2 + gc * (a.conj().T @ sm + a @ sm.conj().T)).tocsr()
    S = math.sqrt(kap) * a
    X = (S + S.conj().T).tocsr()
    k = np.arange(N)
    coh = np.exp(-alpha ** 2 / 2) * alpha ** k / np.sqrt([math.factorial(int(q)) for q in k])
    psi0 = np.kron(coh / np.linalg.norm(coh), np.array([1.0, 0.0]))
    tl = np.linspace(0, 10 * math.pi / wc, 400)
    g = qtl.System(H, [S], [X])
    o = qtl.make_opts(fixed_dt=1e-3)
    for _ in range(args.warmup):
        g.ssesolve(psi0, tl, ntraj, 1, fixed_dt=1e-3)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qtl.launch_count()
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = qtl.ssesolve(g.handle, 1, 1, psi0, tl, ntraj, 1, o)
        ms.append(1e3 * (time.perf_counter() - t0))
    clk = clocks.stop()
    launches = qtl.launch_count() - l0
    g.free()
    mean_ms = statistics.mean(ms)
    t0 = time.perf_counter()
    ref = o_sse(H, [S], [X], psi0, tl, 1e-3, 2, 1)
    t_cpu = time.perf_counter() - t0
    print(json.dumps({
        "metric": "ssesolve traj/s (homodyne JC of Sec. 3.5, 500 trajectories)", "value": ntraj / (mean_ms / 1e3),
        "unit": "traj/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ssesolve_jc: N=20 x 2, wc=wq=5, g=0.1, S=sqrt(1) a, alpha=2, t in [0, 2 pi], 400 saveat, dt 1e-3",
                   "timing": "host API call, host buffers, copies included"},
        "steps_per_traj": r["stats"]["steps_acc"] / ntraj, "X_final": float(r["expect"][0, -1].real),
        "cpu_baseline": {"value": 2 / t_cpu, "unit": "traj/s", "cores": 1, "kind": "oracle",
                         "sample": "oracle ssesolve of 2 trajectories (%.1f s)" % t_cpu},
        "gpu_launches": launches, "clocks": clk}))


def run_smesolve(args):
    """Homodyne stochastic master equation (Sec. 3.5, the paper's example):
    the JC system of the ssesolve workload (N = 20, wc = wq = 5, g = 0.1,
    psi0 = |alpha = 2, e>) with qubit decay sqrt(gamma) sm (gamma = 2) and
    cavity dephasing sqrt(kappa_phi) a^dag a (kappa_phi = 0.3) unmeasured,
    homodyne detection of sqrt(kappa) a (kappa = 1), e_ops {X}, tlist =
    range(0, 10 pi / wc, 400), 500 trajectories, Euler-Maruyama dt = 1e-3,
    FP64.  Value: trajectories per second; the oracle is timed on 1
    trajectory."""
    import math
    import scipy.sparse as sp
    import torch
    from paper_2504_21440_gb300 import qtl
    from oracle.stochastic import smesolve as o_sme
    torch.cuda.set_device(0)
    qtl.load()
    N, wc, wq, gc, kap, gam, kphi, alpha, ntraj = 20, 5.0, 5.0, 0.1, 1.0, 2.0, 0.3, 2.0, 500

    def destroy(M):
        return sp.diags(np.sqrt(np.arange(1, M)), 1, format="csr", dtype=complex)
    a = sp.kron(destroy(N), sp.identity(2), format="csr")
    sm = sp.kron(sp.identity(N), sp.csr_matrix(np.array([[0, 0], [1, 0]], dtype=complex)), format="csr")
    sz = sp.kron(sp.identity(N), sp.csr_matrix(np.diag([1.0, -1.0]).astype(complex)), format="csr")
    H = (wc * a.conj().T @ a + wq * sz / 2 + gc * (a.conj().T @ sm + a @ sm.conj().T)).tocsr()
    C = [math.sqrt(gam) * sm, (math.sqrt(kphi) * a.conj().T @ a).tocsr()]
    S = math.sqrt(kap) * a
    X = (S + S.conj().T).tocsr()
    k = np.arange(N)
    coh = np.exp(-alpha ** 2 / 2) * alpha ** k / np.sqrt([math.factorial(int(q)) for q in k])
    psi0 = np.kron(coh / np.linalg.norm(coh), np.array([1.0, 0.0]))
    tl = np.linspace(0, 10 * math.pi / wc, 400)
    g = qtl.System(H, C + [S], [X])
    o = qtl.make_opts(fixed_dt=1e-3)
    for _ in range(args.warmup):
        qtl.smesolve(g.handle, 1, 1, psi0, tl, ntraj, 1, o)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qtl.launch_count()
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = qtl.smesolve(g.handle, 1, 1, psi0, tl, ntraj, 1, o)
        ms.append(1e3 * (time.perf_counter() - t0))
    clk = clocks.stop()
    launches = qtl.launch_count() - l0
    g.free()
    mean_ms = statistics.mean(ms)
    t0 = time.perf_counter()
    o_sme(H, C, [S], [X], psi0, tl, 1e-3, 1, 1)
    t_cpu = time.perf_counter() - t0
    print(json.dumps({
        "metric": "smesolve traj/s (homodyne JC with losses, Sec. 3.5, 500 trajectories)",
        "value": ntraj / (mean_ms / 1e3), "unit": "traj/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "smesolve_jc: N=20 x 2, wc=wq=5, g=0.1, C={sqrt(2) sm, sqrt(0.3) a'a}, S=a, alpha=2, t in [0, 2 pi], 400 saveat, dt 1e-3",
                   "timing": "host API call, host buffers, copies included"},
        "steps_per_traj": r["stats"]["steps_acc"] / ntraj, "X_final": float(r["expect"][0, -1].real),
        "cpu_baseline": {"value": 1 / t_cpu, "unit": "traj/s", "cores": 1, "kind": "oracle",
                         "sample": "oracle smesolve of 1 trajectory (%.1f s)" % t_cpu},
        "gpu_launches": launches, "clocks": clk}))


# workloads that shard over torchrun ranks; the others run on one GPU
SHARDED = ("jc_40x2", "kerr_sweep_1024")


def main():
    args = parse()
    if args.workload == "ising_c2":
        if args.impl == "reference":
            run_c2_reference(args)
        else:
            run_c2(args)
        return
    if args.impl == "reference" and args.workload != "jc_40x2":
        # the other workloads time the oracle in their own cpu_baseline entry
        sys.exit("bench.py: --impl reference times the ising_c2 and jc_40x2 jobs; the line of --workload %s "
                 "carries its own oracle timing (cpu_baseline)" % args.workload)
    if args.workload not in SHARDED and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        sys.exit("bench.py: --workload %s runs on one GPU (no torchrun)" % args.workload)
    if args.workload == "smesolve_jc" and args.impl != "reference":
        run_smesolve(args)
        return
    if args.workload == "ssesolve_jc" and args.impl != "reference":
        run_ssesolve(args)
        return
    if args.workload == "optomech_td" and args.impl != "reference":
        run_optomech(args)
        return
    if args.workload == "steadystate" and args.impl != "reference":
        run_steady(args)
        return
    if args.workload == "dsf_mc" and args.impl != "reference":
        run_dsf_mc(args)
        return
    if args.workload == "dsf" and args.impl != "reference":
        run_dsf(args)
        return
    if args.workload == "serving" and args.impl != "reference":
        run_serving(args)
        return
    if args.workload == "ising10" and args.impl != "reference":
        run_ising10(args)
        return
    if args.workload == "ising14_mc" and args.impl != "reference":
        run_ising14_mc(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "kerr_sweep_1024":
        run_sweep(args)
    else:
        run_qtl(args)


if __name__ == "__main__":
    main()
