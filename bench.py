"""Benchmark of the fused reactive-mixture lattice Boltzmann step on GB300.

Workload: the 3D expanding-flame configuration, a periodic 256^3 D3Q27
lattice with the nine-species, 21-reaction seeded mechanism, T = 300 K and
a 2000 K spherical kernel of radius 20 (seeded composition noise), mixed
precision (float populations; double temperature iteration, Stefan-Maxwell
solve and chemistry).  The same lattice is also stepped with the double
path for the mixed/double ratio.  One "step" is one full time step of every
node (ghost/moment/gradient/collision kernels).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
instead (a bounded sample of the same physics on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MLUPS (M+2 pop sets + chemistry), mixed vs FP64 step, % of HBM roofline"
FALLBACK_HBM_GBS = 6800.0

# FP64 arithmetic peak derived from the unit counts: 152 SMs x 2 FP64 FMA
# per SM and clock x 2 flops x 2070 MHz (maximum SM clock).  The roofline
# uses the peak measured by lbm_fp64_probe on the same GPU in the same run;
# the derived figure is reported beside it.
SM_COUNT, FP64_FMA_PER_SM_CLK, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_TFLOPS_DERIVED = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12

# Per lattice node and launch, counted by ncu for the kernels as they
# stand (profiles/ has the captures and their commands):
#   FP64 flops = 2 x DFMA + DADD + DMUL thread instructions (64^3 instance:
#   instruction counts per node do not depend on the lattice size);
#   DRAM bytes = dram__bytes_read.sum + dram__bytes_write.sum on the 256^3
#   lattice itself (a smaller one keeps part of its state in L2).
# The production rates are formed inside k_step (no k_chem launch), so
# their flops count there.
FP64_FLOPS_PER_NODE = {
    "mixed": {"k_pre": 1873.6, "k_step_g": 165.0, "k_step": 1189.0},
    "mixed_fast": {"k_pre": 621.5, "k_step_g": 165.0, "k_step": 663.0},
    "fp64": {"k_pre": 2561.6, "k_step_g": 737.0, "k_step": 13688.0},
}
# lbm_heat_release (k_hrr: moments, temperature, hdot^c and its derivatives
# per node), counted the same way; None until counted.
HRR_FLOPS_PER_NODE = {"mixed": 3123.0, "mixed_fast": None, "fp64": None}
DRAM_BYTES_PER_NODE = {
    "mixed": {"k_pre": 2165.2, "k_step_g": 617.3, "k_step": 2438.2},
    "mixed_fast": {"k_pre": 2275.2, "k_step_g": 600.5, "k_step": 2398.0},
    "fp64": {"k_pre": 3415.9, "k_step_g": 699.7, "k_step": 4458.0},
}


def launches_per_step(ghost: bool) -> int:
    """Kernels one step launches: moments, gradients, energy and species
    collisions (the production rates are formed inside the species
    collision), plus the ghost-node kernel for non-periodic x."""
    return 4 + (1 if ghost else 0)


def algorithmic_bytes_per_node(M: int, mixed: bool) -> int:
    """One read and one write of the (M+1) stored sets of 27 populations,
    4 bytes each in mixed precision and 8 in double: 2160 and 4320 B at
    M = 9.  The mixed layout moves a little more (stored_bytes_per_node:
    double rest populations and a double energy set)."""
    return 2 * (M + 1) * 27 * (4 if mixed else 8)


def fp64_probe(lbm, torch, stream, blocks_per_sm: int = 8):
    """Measured double-precision throughput of this GPU (lbm_fp64_probe):
    fused multiply-add in TFLOP/s, CUDA's exp and log in G calls/s, each a
    single launch of 152 x blocks_per_sm blocks of 256 threads timed with
    CUDA events after a short warm-up launch."""
    blocks = SM_COUNT * blocks_per_sm
    sink = torch.zeros(blocks, dtype=torch.float64, device=stream.device)
    out = {}
    for name, kind, iters in (("dfma", lbm.LBM_PROBE_DFMA, 24000), ("exp", lbm.LBM_PROBE_EXP, 3000),
                              ("log", lbm.LBM_PROBE_LOG, 3000)):
        st, _, _ = lbm.lbm_fp64_probe(kind, blocks, max(1, iters // 50), sink.data_ptr(), stream.cuda_stream)
        if st != lbm.LBM_OK:
            raise lbm.LBMError(st, "lbm_fp64_probe")
        st, ms, rate = lbm.lbm_fp64_probe(kind, blocks, iters, sink.data_ptr(), stream.cuda_stream)
        if st != lbm.LBM_OK:
            raise lbm.LBMError(st, "lbm_fp64_probe")
        out[name] = {"ms": ms, "rate": rate}
    return {"dfma_tflops": out["dfma"]["rate"] / 1e12, "exp_gcalls": out["exp"]["rate"] / 1e9,
            "log_gcalls": out["log"]["rate"] / 1e9,
            "ms": {k: v["ms"] for k, v in out.items()},
            "derived_tflops": FP64_PEAK_TFLOPS_DERIVED,
            "how": f"lbm_fp64_probe: {blocks} blocks x 256 threads; 8 independent FMA chains per thread "
                   f"(2 flop each), 4 independent exp / log chains per thread; CUDA events"}


def adjoint_timing(lbm, torch, steps: int = 2000, every: int = 64, nx: int = 512):
    """Gradients of the time-integrated heat release through the dynamics on
    the periodic quasi-1D flame (nx x 4 x 4, nine species, double): the
    objective alone (forward sweep) against the objective with dJ/d ln A_k
    and dJ/dT(x, 0) (forward sweep with checkpoints, reverse sweep with
    recomputation), host-timed around calls that end with a stream wait;
    peak device memory of the solver and workspace."""
    import workload as w
    prob = w.adjoint_flame_problem(nx=nx)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.heat_release_gradient(8, 4)                               # warm-up of every kernel
    s.init(prob.init.X, prob.init.T, None, prob.init.P)
    t0 = time.perf_counter()
    J_fwd = s.heat_release_total(steps)
    t_fwd = time.perf_counter() - t0
    s.init(prob.init.X, prob.init.T, None, prob.init.P)
    t0 = time.perf_counter()
    J, dA, dT0, ws = s.heat_release_gradient(steps, every)
    t_all = time.perf_counter() - t0
    peak = torch.cuda.max_memory_allocated() - base
    gT = dT0.abs().max().item()
    s.close()
    del s, dT0
    torch.cuda.empty_cache()
    return {"workload": prob.name, "nodes": prob.lattice.n_nodes, "steps": steps, "checkpoint_every": every,
            "forward_s": t_fwd, "forward_and_backward_s": t_all, "backward_over_forward": (t_all - t_fwd) / t_fwd,
            "peak_device_bytes": int(peak), "workspace_bytes": int(ws), "J": J, "J_forward_only": J_fwd,
            "max_abs_dJ_dlogA": float(np.abs(dA).max()), "max_abs_dJ_dT0": gT,
            "note": "lbm_heat_release_gradient: J = sum over steps and nodes of hdot^c; gradients with respect "
                    "to the 21 ln A_k and T(x, 0); FP64"}


def circular_flame_run(lbm, torch, stream, precision, n: int = 512, steps: int = 2000, every: int = 250):
    """The perturbed circular expanding flame of Sec. 5b (Eq. (cflamePerturbation),
    R_ig = 48, A0 = 0.05, n0 = 4) on a periodic n x n x 1 box: every `every`
    steps the mean radius of the T = 3 T_u isoline (Eq. (rmean)) and the
    isoline means of S_a and of rho S_d / rho_u (Eq. (sd)), from
    lbm_flame_speeds and lbm_isoline_means; the time of the diagnostics."""
    import workload as w
    prob = w.circular_flame_problem(n=n, R_ig=48.0, A0=0.05, n0=4)
    s = lbm.Solver.from_problem(prob, precision=precision, stream=stream)
    c = (n - 1) / 2.0
    T_u = 298.0
    rec = []
    t_diag = 0.0
    t = 0
    while True:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = s.moments(lbm.LBM_F_T | lbm.LBM_F_RHO_A, device=True)
        Sd, Sa = s.flame_speeds(device=True)
        rho = m["rho_a"].sum(dim=0)
        rho_u = float(rho[0].item())                  # a corner node: unburnt
        out = s.isoline_means(m["T"], 3 * T_u, c, c, [Sa, rho * Sd / rho_u])
        torch.cuda.synchronize()
        t_diag += time.perf_counter() - t0
        rec.append({"step": t, "length": out[0], "R_mean": out[1], "S_a": out[2], "S_d_hat": out[3]})
        del m, Sd, Sa, rho
        if t >= steps:
            break
        s.step(every)
        t += every
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"workload": prob.name, "isoline": "T = 3 T_u", "samples": rec,
            "diagnostics_ms": 1e3 * t_diag / len(rec),
            "note": "lattice units; quasi-2D periodic box (the paper's quarter domain with symmetry and "
                    "characteristic outlets is not built); burnt region of the unburnt composition at T_b"}


def stored_bytes_per_node(M: int, mixed: bool) -> int:
    """Bytes of one copy of the stored state per node: in mixed precision the
    26 moving populations of the M species/mixture sets in float, their rest
    populations and the 27 energy populations in double; otherwise all
    (M+1) x 27 populations in double."""
    return M * 26 * 4 + M * 8 + 27 * 8 if mixed else (M + 1) * 27 * 8


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_oracle_sample(min_seconds: float = 10.0, max_steps: int = 400, warmup: int = 1):
    """The FP64 oracle on the 32^3 instance of the same physics (radius-8
    kernel), timed on all host cores."""
    import oracle
    import workload as w
    prob = w.sphere3d_problem(n=32, radius=8.0)
    o = oracle.Oracle.from_problem(prob)
    o.step(warmup)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps and (time.perf_counter() - t0) < min_seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 32 ** 3 * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"sphere3d 32^3 (radius 8), 9 species / 21 reactions, FP64, {n} steps in {dt:.1f} s"}


def _cpu_oracle_single_thread(min_seconds: float = 3.0):
    """The same sample on one host thread (a child process started with
    OMP_NUM_THREADS=1, so that this process's thread pool is untouched)."""
    code = ("import json, bench; r = bench._cpu_oracle_sample(min_seconds=%r, max_steps=100); "
            "print(json.dumps(r))" % min_seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=str(ROOT), env=env, capture_output=True, text=True,
                       timeout=120)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_leg(prob, steps: int, warmup: int = 1):
    """The FP64 oracle stepping one whole workload on all host cores."""
    import oracle
    o = oracle.Oracle.from_problem(prob)
    o.step(warmup)
    t0 = time.perf_counter()
    assert o.step(steps) == 0
    dt = time.perf_counter() - t0
    N = prob.lattice.n_nodes
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "seconds": dt, "steps": steps,
            "nodes": N, "workload": prob.name}


def _host_memory_bytes():
    """Memory this process may still use: MemAvailable, capped by a cgroup limit."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for f in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            v = open(f).read().strip()
            if v.isdigit():
                avail = min(avail or int(v), int(v))
        except OSError:
            pass
    return avail


def run_cpu_legs(args):
    """The oracle's three timed legs: the three-gas 64x4x4 workload for 200
    steps, the 32^3 expanding flame for 1000 steps, and 10 steps of the
    256^3 benchmark lattice (only when the host has memory for the oracle's
    ~5.1 kB per node, with half again to spare)."""
    import workload as w
    legs = {"config1_64x4x4_M3_200": _cpu_leg(w.config1_problem(), 200),
            "sphere3d_32^3_M9_1000": _cpu_leg(w.sphere3d_problem(n=32, radius=8.0), 1000)}
    need = 256 ** 3 * 5200
    have = _host_memory_bytes()
    if have is not None and have > 1.5 * need:
        legs["sphere3d_256^3_M9_10"] = _cpu_leg(w.sphere3d_problem(n=256, radius=20.0), 10)
    else:
        legs["sphere3d_256^3_M9_10"] = {"skipped": f"needs ~{need / 1e9:.0f} GB of host memory, "
                                                   f"{(have or 0) / 1e9:.0f} GB available"}
    print(json.dumps({"metric": "FP64 CPU oracle MLUPS per leg", "legs": legs}), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workload as w
    prob = w.sphere3d_problem(n=32, radius=8.0)
    o = oracle.Oracle.from_problem(prob)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = 32 ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "sphere3d_32^3_M9_fp64 (bounded sample of sphere3d_256^3_M9)",
                       "nodes": 32 ** 3, "species": 9, "reactions": 21},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"sphere3d 32^3 (radius 8), FP64, {args.steps} steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import workload as w
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm, replicas

    n = args.size
    prob = w.sphere3d_problem(n=n, radius=20.0 * n / 256.0)
    N = prob.lattice.n_nodes
    M = prob.species.M
    S = M + 1
    modes = {"mixed": lbm.LBM_MIXED, "mixed_fast": lbm.LBM_MIXED_FAST, "fp64": lbm.LBM_FP64}
    precision = modes[args.precision]
    stream = torch.cuda.Stream()

    def timed_steps(solver, K):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        solver.step_async(K)
        e1.record(stream)
        st = solver.sync()
        torch.cuda.synchronize()
        barrier()
        if st != lbm.LBM_OK:
            raise lbm.LBMError(st, "timed steps")
        return e0.elapsed_time(e1)

    # ---- device-resident run (value) ------------------------------------
    # The timed region: K steps enqueued back to back on the library's
    # stream with CUDA events between the kernels (one wait at the end);
    # the events give the whole-run time and each kernel's launch times.
    with ClockSampler(local) as clk_probe:
        probe = fp64_probe(lbm, torch, stream)                     # the FP64 peak, before the timed region
    probe["clocks"] = clk_probe.summary()
    FP64_PEAK = probe["dfma_tflops"]
    s = lbm.Solver.from_problem(prob, precision=precision, stream=stream)
    blocks = None if args.skip_autotune else s.autotune(trials=3)   # launch shapes, outside the timed region
    s.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        ph = s.step_timed(args.steps)
    torch.cuda.synchronize()
    barrier()
    ms = float(ph[lbm.LBM_PHASES])
    phases = ph[:lbm.LBM_PHASES] / args.steps            # ms per launch: ghost, pre, chem, grad, step_g, step
    ms = replicas.max_over_ranks(ms, dist, "cuda")        # the job is as slow as its slowest replica
    mlups = replicas.whole_job_mlups([N] * world, args.steps, ms)

    # ---- rooflines --------------------------------------------------------
    # The step is bound by FP64 arithmetic (temperature iteration, energy
    # moments, reaction rates): the roofline of the longest kernel is the
    # FP64 one.  The HBM view of the whole step counts one read and one write
    # of the stored state per node.
    peak, peak_kind = _peaks()
    mixed = precision != lbm.LBM_FP64
    alg_bytes_node = algorithmic_bytes_per_node(M, mixed)
    layout_bytes_node = 2 * stored_bytes_per_node(M, mixed)
    step_frac = alg_bytes_node * N / (ms * 1e-3 / args.steps) / 1e9 / peak
    kern_ms = {"k_pre": phases[1], "k_chem": phases[2], "k_grad": phases[3], "k_step_g": phases[4],
               "k_step": phases[5]}
    del kern_ms["k_chem"]                              # fused into k_step
    flops = FP64_FLOPS_PER_NODE[args.precision]
    dram = DRAM_BYTES_PER_NODE[args.precision]
    kernels = {}
    for k, t in kern_ms.items():
        e = {"ms": t}
        if flops.get(k):
            e["fp64_tflops"] = flops[k] * N / (t * 1e-3) / 1e12
            e["fp64_frac"] = e["fp64_tflops"] / FP64_PEAK
        if dram.get(k):
            e["dram_gbs"] = dram[k] * N / (t * 1e-3) / 1e9
        kernels[k] = e
    dom = max((k for k in ("k_pre", "k_chem", "k_step_g", "k_step") if k in kern_ms), key=lambda k: kern_ms[k])
    roofline = {"bound": "alu", "kernel": dom, "achieved": kernels[dom].get("fp64_tflops"),
                "peak": FP64_PEAK, "unit": "TFLOP/s", "frac": kernels[dom].get("fp64_frac"),
                "traffic": dram[dom] * N if dram.get(dom) else None,
                "flops_per_node": flops.get(dom),
                "peak_source": "measured: lbm_fp64_probe DFMA throughput in this run (of measured)",
                "frac_of_derived_peak": (kernels[dom]["fp64_tflops"] / FP64_PEAK_TFLOPS_DERIVED
                                         if kernels[dom].get("fp64_tflops") else None)}
    roofline_hbm = {"bound": "hbm", "kernel": "whole step",
                    "achieved": alg_bytes_node * N / (ms * 1e-3 / args.steps) / 1e9, "peak": peak,
                    "unit": "GB/s", "frac": step_frac, "algorithmic_bytes_per_node": alg_bytes_node,
                    "layout_bytes_per_node": layout_bytes_node,
                    "layout_frac": layout_bytes_node * N / (ms * 1e-3 / args.steps) / 1e9 / peak,
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}

    # ---- heat-release objective and its sensitivities ---------------------
    # lbm_heat_release on the state the timed steps left: hdot^c summed over
    # the lattice, dJ/d ln A_k, and the per-node derivatives in T and rho_a
    # (device outputs).  Outside the timed step region.
    hrr = None
    if not args.skip_hrr:
        dT = torch.empty(N, dtype=torch.float64, device=stream.device)
        dr = torch.empty((M, N), dtype=torch.float64, device=stream.device)
        J = np.zeros(1)
        dA = np.zeros(prob.mech.R)

        def hrr_call():
            st = lbm.lbm_heat_release(s.ctx, J, dA, dT.data_ptr(), dr.data_ptr())
            if st != lbm.LBM_OK:
                raise lbm.LBMError(st, "lbm_heat_release")

        hrr_call()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            hrr_call()
        e1.record(stream)
        torch.cuda.synchronize()
        t_hrr = e0.elapsed_time(e1) / reps
        hrr = {"ms": t_hrr, "mnodes_per_s": N / (t_hrr * 1e-3) / 1e6, "J": float(J[0]),
               "outputs": "J, dJ/dlnA_k (R), d hdot/dT (N), d hdot/d rho_a (M x N) on the device"}
        f_h = HRR_FLOPS_PER_NODE.get(args.precision)
        if f_h:
            hrr["fp64_tflops"] = f_h * N / (t_hrr * 1e-3) / 1e12
            hrr["fp64_frac"] = hrr["fp64_tflops"] / FP64_PEAK
            hrr["flops_per_node"] = f_h
        del dT, dr
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers ------------------
    e2e = None
    if not args.skip_e2e:
        Xh = torch.from_numpy(prob.init.X).pin_memory()
        Th = torch.from_numpy(prob.init.T).pin_memory()
        mask = lbm.LBM_F_T | lbm.LBM_F_Y
        out = torch.empty(lbm.lbm_moments_count(s.ctx, mask), dtype=torch.float64).pin_memory()
        runs, parts = [], []
        for _ in range(3):                     # the whole job three times; the median is reported
            torch.cuda.synchronize()
            barrier()
            # each call returns after its stream has drained, so the host
            # clock between them splits the run into its three parts
            t0 = time.perf_counter()
            st = lbm.lbm_init(s.ctx, Xh.data_ptr(), Th.data_ptr(), None, prob.init.P)
            t1 = time.perf_counter()
            for _ in range(args.steps):        # each step reads its status word back to the host
                st = st or lbm.lbm_step(s.ctx, 1)
            t2 = time.perf_counter()
            st = st or lbm.lbm_moments(s.ctx, mask, out.data_ptr())
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            barrier()
            if st != lbm.LBM_OK:
                raise lbm.LBMError(st, "e2e")
            runs.append(N * args.steps * world / (t3 - t0) / 1e6)
            parts.append({"init_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3, "moments_out_ms": (t3 - t2) * 1e3})
        h2d = (M + 1) * N * 8
        d2h = out.numel() * 8 + 4 * args.steps
        e2e = {"value": statistics.median(runs), "unit": "MLUPS", "runs": runs, "parts": parts,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "lbm_init from pinned host fields, then each step with its status word read back, "
                       "then lbm_moments(T, Y) to pinned host; median of three whole runs"}
    s.close()
    del s
    torch.cuda.empty_cache()

    # ---- the fast mixed mode on the same lattice ---------------------------
    fast = None
    if not args.skip_fast and precision == lbm.LBM_MIXED:
        sf = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED_FAST, stream=stream)
        sf.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        phf = sf.step_timed(args.steps)
        torch.cuda.synchronize()
        barrier()
        msf = float(phf[lbm.LBM_PHASES])
        phf = phf[:lbm.LBM_PHASES] / args.steps
        fast = {"mlups": N * args.steps * world / (msf * 1e-3) / 1e6, "steps": args.steps,
                "phase_ms": {"moments": phf[1], "chemistry": phf[2], "gradients": phf[3],
                             "energy_collision": phf[4], "species_collision": phf[5]},
                "note": "LBM_MIXED_FAST: Stefan-Maxwell solve and relaxation in float, exponentials of the "
                        "rates with a float 2^f; same storage and accuracy bar"}
        sf.close()
        del sf
        torch.cuda.empty_cache()

    # ---- mixture-averaged transport (viscosity, conductivity and
    # diffusivities of each node's state) on the same lattice ---------------
    transport = None
    if not args.skip_fast and precision == lbm.LBM_MIXED:
        pt = w.sphere3d_problem(n=n, radius=20.0 * n / 256.0)
        pt.species = w.with_mixture_transport(pt.species, w.configs.PHI1_X + 1e-12, pt.mech.P0, 300.0)
        st_ = lbm.Solver.from_problem(pt, precision=lbm.LBM_MIXED, stream=stream)
        st_.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        pht = st_.step_timed(args.steps)
        torch.cuda.synchronize()
        barrier()
        mst = float(pht[lbm.LBM_PHASES])
        pht = pht[:lbm.LBM_PHASES] / args.steps
        transport = {"mlups": N * args.steps * world / (mst * 1e-3) / 1e6, "steps": args.steps,
                     "phase_ms": {"moments": pht[1], "gradients": pht[3], "energy_collision": pht[4],
                                  "species_collision": pht[5]},
                     "note": "LBM_MIXED with LBM_TRANSPORT_MIXTURE_AVERAGED (Wilke viscosity, Eucken/Mathur "
                             "conductivity, power-law diffusivities per node)"}
        st_.close()
        del st_
        torch.cuda.empty_cache()

    # ---- the double-precision step on the same lattice -------------------
    fp64 = None
    if not args.skip_fp64 and precision == lbm.LBM_MIXED:
        s64 = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64, stream=stream)
        s64.step(max(1, args.warmup // 2))
        k64 = max(2, args.steps // 2)
        ms64 = timed_steps(s64, k64)
        fp64 = {"mlups": N * k64 * world / (ms64 * 1e-3) / 1e6, "steps": k64,
                "hbm_frac": algorithmic_bytes_per_node(M, False) * N / (ms64 * 1e-3 / k64) / 1e9 / peak}
        s64.close()
        del s64
        torch.cuda.empty_cache()

    adjoint = None
    if not args.skip_adjoint:
        adjoint = adjoint_timing(lbm, torch)

    cflame = None
    if not args.skip_cflame:
        cflame = circular_flame_run(lbm, torch, stream, precision)

    flames48 = None
    if not args.skip_flames:
        flames48 = flames_measure(lbm, w, replicas, precision, args.flames_steps, args.warmup, stream, dist, rank,
                                  world, autotune=not args.skip_autotune)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = _cpu_oracle_sample()
        one = _cpu_oracle_single_thread()
        if one:
            cpu["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
        cpu["legs"] = {"config1_64x4x4_M3_200": _cpu_leg(w.config1_problem(), 200)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
            "config": {"workload": f"sphere3d_{n}^3_M9_{args.precision}", "nodes": N, "species": M,
                       "reactions": prob.mech.R, "stored_sets": S, "precision": args.precision,
                       "parallelism": f"replicas{world}" if world > 1 else "single_gpu",
                       "l2": "inputs larger than L2 (state %.1f GB per copy)"
                             % (stored_bytes_per_node(M, mixed) * N / 1e9)},
            "hbm_frac_step": step_frac,
            "phase_ms": {"ghost": phases[0], "moments": phases[1], "chemistry": phases[2],
                         "gradients": phases[3], "energy_collision": phases[4], "species_collision": phases[5]},
            "roofline": roofline,
            "roofline_hbm": roofline_hbm,
            "fp64_peak_measured": probe,
            "kernels": kernels,
            "autotuned_blocks": blocks,
            "mixed_fast_step": fast,
            "mixture_averaged_transport_step": transport,
            "fp64_step": fp64,
            "heat_release": hrr,
            "adjoint": adjoint,
            "circular_flame": cflame,
            "flames48": flames48,
            "mixed_over_fp64": (mlups / fp64["mlups"]) if fp64 else None,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step(prob.lattice.bc_x != 0),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def flames_measure(lbm, w, replicas, precision, K, warmup, stream, dist=None, rank=0, world=1,
                   autotune=True, clk=None):
    """The batched quasi-1D flames (48 ragged flames side by side in one
    lattice) stepped K times three ways -- one set of launches per step,
    those launches replayed from a captured CUDA graph, and one persistent
    cooperative launch for all K steps -- against the same flames stepped
    one flame at a time (one context per flame, sharing the batch's
    tables).  With N ranks the flames are split across them by node count
    (no collective on the data path); MLUPS count all ranks' nodes over the
    slowest rank."""
    import torch
    L_all, phi_all = w.batched_flames_lengths()
    shards = replicas.shard_lengths(L_all, world)
    mine = shards[rank]
    prob = w.batched_flames_problem(lengths=[L_all[k] for k in mine], phis=[phi_all[k] for k in mine])

    def timed(fn):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        return replicas.max_over_ranks(e0.elapsed_time(e1), dist, "cuda")

    batch = lbm.Solver.from_problem(prob, precision=precision, stream=stream)
    # launch shapes and the persistent tile length, outside the timed region
    blocks = batch.autotune(trials=3) if autotune else None
    tile = batch.autotune_persistent(steps=4) if autotune else 1
    batch.step(warmup)
    batch.step_persistent(warmup, tile_mult=tile)
    ms_plain = timed(lambda: batch.step_async(K))
    batch.step_graph(2)                           # capture outside the timed region
    assert batch.sync() == lbm.LBM_OK
    ms_graph = timed(lambda: batch.step_graph(K))
    assert batch.sync() == lbm.LBM_OK
    ms_pers = timed(lambda: batch.step_persistent(K, tile_mult=tile))
    T = batch.moments(lbm.LBM_F_T)["T"]
    finite = bool(np.isfinite(T).all())
    refs = batch.references() if precision != lbm.LBM_FP64 else None
    batch.close()
    del batch
    torch.cuda.empty_cache()

    flames = []
    for k in range(len(prob.lattice.seg_nx)):
        fk = w.flame_of_batch(prob, k)
        s = lbm.Solver.from_problem(fk, precision=precision, stream=stream, init=False)
        if refs is not None:
            s.set_references(refs)
        s.init(fk.init.X, fk.init.T, fk.init.u, fk.init.P)
        s.step(warmup)
        flames.append(s)

    def loop():
        for _ in range(K):
            for s in flames:
                s.step_async(1)
    ms_loop = timed(loop)
    for s in flames:
        assert s.sync() == lbm.LBM_OK
        s.close()

    nodes = [sum(int(L_all[k]) for k in shards[r]) * prob.lattice.ny * prob.lattice.nz for r in range(world)]
    mlups = lambda ms: replicas.whole_job_mlups(nodes, K, ms)
    best = min(("graph", ms_graph), ("persistent", ms_pers), key=lambda t: t[1])
    return {"workload": f"flames{len(L_all)}_M9", "nodes": sum(nodes), "flames": len(L_all),
            "lengths": [int(min(L_all)), int(max(L_all))], "cross_section": "4x4", "steps": K,
            "persistent_mlups": mlups(ms_pers), "batched_graph_mlups": mlups(ms_graph),
            "batched_plain_mlups": mlups(ms_plain), "loop_single_flames_mlups": mlups(ms_loop),
            "best": best[0], "best_mlups": mlups(best[1]), "speedup_vs_loop": ms_loop / best[1],
            "persistent_over_graph": ms_graph / ms_pers, "persistent_chunk_nodes": 32 * tile,
            "autotuned_blocks": blocks, "temperature_finite": finite,
            "ms": {"plain": ms_plain, "graph": ms_graph, "persistent": ms_pers, "loop": ms_loop},
            "launches": {"plain": K * launches_per_step(True), "graph": K * launches_per_step(True),
                         "persistent": 1, "loop": K * len(prob.lattice.seg_nx) * launches_per_step(True)}}


def run_flames(args):
    """The batched flames as a line of their own (see flames_measure); the
    value is the faster of the graph and the persistent launch."""
    import torch
    import workload as w
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm, replicas

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    modes = {"mixed": lbm.LBM_MIXED, "mixed_fast": lbm.LBM_MIXED_FAST, "fp64": lbm.LBM_FP64}
    precision = modes[args.precision]
    stream = torch.cuda.Stream()
    with ClockSampler(local) as clk:
        r = flames_measure(lbm, w, replicas, precision, args.steps, args.warmup, stream, dist, rank, world,
                           autotune=not args.skip_autotune)
    K = args.steps
    if rank == 0:
        line = {"metric": "MLUPS (batched quasi-1D flames)", "value": r["best_mlups"],
                "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": args.warmup,
                "ms_per_step": r["ms"][r["best"]] / K, "higher_is_better": True,
                "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
                "dtype": "f32+f64" if precision != lbm.LBM_FP64 else "f64", "data": "synthetic",
                "config": {"workload": f"{r['workload']}_{args.precision}", "nodes": r["nodes"],
                           "flames": r["flames"], "lengths": r["lengths"], "cross_section": "4x4",
                           "parallelism": f"flames split over {world} ranks" if world > 1 else "single_gpu"},
                "flames48": r,
                "gpu_launches": r["launches"][r["best"]],
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_accuracy(args):
    """Field error of the mixed modes against the double GPU step on the
    whole benchmark lattice after K steps: max |F - F_fp64| / max |F_fp64|
    for T and for each Y_a (the 1e-4 bar of the mixed-precision design).
    The three runs advance side by side, so --accuracy-every E also records
    the errors every E steps (the growth of the error in time)."""
    import torch
    import workload as w
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm

    n = args.size
    prob = w.sphere3d_problem(n=n, radius=20.0 * n / 256.0)
    K = args.accuracy_steps
    every = args.accuracy_every if args.accuracy_every > 0 else K
    mask = lbm.LBM_F_T | lbm.LBM_F_Y
    modes = (("fp64", lbm.LBM_FP64), ("mixed", lbm.LBM_MIXED), ("mixed_fast", lbm.LBM_MIXED_FAST))
    solvers = {name: lbm.Solver.from_problem(prob, precision=p) for name, p in modes}
    seconds = {name: 0.0 for name, _ in modes}
    history = []
    done = 0
    out = {"metric": f"relative field error after {K} steps against the double GPU step",
           "config": {"workload": f"sphere3d_{n}^3_M9", "nodes": prob.lattice.n_nodes, "steps": K}}
    while done < K:
        k = min(every, K - done)
        for name, _ in modes:
            t0 = time.perf_counter()
            solvers[name].step(k)
            seconds[name] += time.perf_counter() - t0
        done += k
        ref = solvers["fp64"].moments(mask, device=True)
        rec = {"step": done}
        for name in ("mixed", "mixed_fast"):
            m = solvers[name].moments(mask, device=True)
            errT = float(((m["T"] - ref["T"]).abs().max() / ref["T"].abs().max()).item())
            errY = [float(((m["Y"][a] - ref["Y"][a]).abs().max() / ref["Y"][a].abs().max()).item())
                    for a in range(prob.species.M)]
            rec[name] = {"T": errT, "Y": errY, "max": max([errT] + errY)}
            del m
        del ref
        torch.cuda.empty_cache()
        history.append(rec)
    for name in ("mixed", "mixed_fast"):
        out[name] = dict(history[-1][name], seconds=seconds[name])
    out["fp64_seconds"] = seconds["fp64"]
    if len(history) > 1:
        out["history"] = [{"step": h["step"], "mixed": h["mixed"]["max"], "mixed_fast": h["mixed_fast"]["max"],
                           "mixed_argmax": max(range(len(h["mixed"]["Y"])), key=lambda a: h["mixed"]["Y"][a])}
                          for h in history]
    for s in solvers.values():
        s.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_fast", "fp64"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-fast", action="store_true")
    ap.add_argument("--skip-autotune", action="store_true", help="keep the default launch shapes (profiling runs)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-hrr", action="store_true", help="skip the heat-release sensitivity measurement")
    ap.add_argument("--skip-adjoint", action="store_true", help="skip the gradients through time (512x4x4, 2000 steps)")
    ap.add_argument("--skip-cflame", action="store_true", help="skip the perturbed circular flame (512x512x1)")
    ap.add_argument("--skip-flames", action="store_true", help="skip the batched-flames key of the default line")
    ap.add_argument("--flames-steps", type=int, default=20, help="steps of the batched-flames key")
    ap.add_argument("--workload", default="sphere3d", choices=["sphere3d", "flames48"])
    ap.add_argument("--cpu-legs", action="store_true",
                    help="instead of timing the GPU: the oracle's timed legs (64x4x4 200 steps, 32^3 1000 steps, "
                         "256^3 10 steps)")
    ap.add_argument("--accuracy-every", type=int, default=0,
                    help="with --accuracy-steps: also record the errors every this many steps")
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="instead of timing: field error of the mixed modes against double after this many steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.cpu_legs:
        run_cpu_legs(args)
    elif args.accuracy_steps > 0:
        run_accuracy(args)
    elif args.workload == "flames48":
        run_flames(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
