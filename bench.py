#!/usr/bin/env python3
"""Throughput of the reduced-Newton MG-MINRES solve of the PBM method (Brune & Kocvara, arXiv:1904.06556).

One step is one complete reduced Newton system of the synthetic workload, every row of the hot path:
  * Newton state set-up (per-element coefficients rho', rho'', mu'', d, eps; the alpha border; the Galerkin
    coarse operators of S on every level; Jacobi diagonals; Lanczos estimates of the smoother weights; the
    Cholesky inverse of the coarsest bordered matrix),
  * the right-hand side of eq. (system),
  * MINRES preconditioned by one V-cycle per iteration, until the true 2-norm relative residual is at most rtol.

Default workload: the 128 x 64 x 64 bridge (four bottom corners fixed, unit top traction, 32-bump density at
volume fraction 0.2, 6-level V-cycle, rtol 1e-8) at its synthetic Newton state, solved with FP32 inner solves inside
FP64 refinement ("mixed", the JSON line's value) and, in the same process on the same inputs, with the plain FP64
solve; both solutions are compared with the oracle's reference solution of the same system
(tests/golden/bridge128_dz_ref.npy, MG-MINRES to about 2e-14, written by tests/golden/make_bridge128_reference.py).
The JSON line reports whole-job solves per second (device-resident inputs, L2 flushed between steps), the same
measured end to end through the C ABI with the inputs copied from pinned host memory and the solution copied back
every step, the roofline of the fine-level FP32 S kernel (timed live by the library with CUDA events on its launch
stream), the clocks sampled during the timed region and the CPU oracle's time for a bounded sample of the same
system.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload bridge128|cant64|...]
                  [--precision mixed|fp64] [--no-compare]

`--impl reference` times the CPU oracle (oracle/, numpy/scipy) on the host cores for the same workload and
metric. With N > 1 (torchrun) every rank solves its own replica of the workload (weak scaling; the solve itself
is not partitioned across GPUs).
"""
from __future__ import annotations

import os

# dense and factorisation parts of the CPU oracle (BLAS) use every host core; scipy's sparse products are
# single-threaded whatever this says
_NCPU = str(os.cpu_count() or 1)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, _NCPU)

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import re  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "reduced-Newton MG-MINRES solve time & K(ρ)u GB/s; FP32-mixed vs FP64"
UNIT = "reduced-Newton solves/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_DIR = os.path.join(ROOT, "profiles")
# source of the fine-level S kernel whose ncu traffic a committed profile may quote, per precision
# the device code of the roofline kernels: the file up to the marker line that starts its host-side part
# (launch wrappers, plans, cost models), so that host-only edits keep the ncu counters valid
KERNEL_SOURCES = {"fp64": [(os.path.join(ROOT, "paper_1904_06556_gb300", "csrc", "colpass.cu"), "// launch wrappers")],
                  "mixed": [(os.path.join(ROOT, "paper_1904_06556_gb300", "csrc", "fused.cu"),
                             "// FP32 coarse levels"),
                            (os.path.join(ROOT, "paper_1904_06556_gb300", "csrc", "strip.cu"),
                             "// plans: element rows per warp"),
                            (os.path.join(ROOT, "paper_1904_06556_gb300", "csrc", "fp32_elem.h"), None)]}
# FP64 issue rate of GB300 derived from the nominal 1.25 TFLOP/s (FMA = 2 flops), 152 SMs, 2070 MHz:
# 1.25e12 / (2 * 152 * 2.07e9) = 2 FP64 instructions per clock per SM, i.e. 629 G FP64 operations/s.
FP64_OPS_PEAK = 2.0 * 152 * 2.07e9
FALLBACK_HBM_GBS = 6800.0


def workload_desc(w, precision, smoother="jacobi", compare=None):
    prec = precision if not compare else f"{precision} (FP32 inner solves in FP64 refinement) vs {compare}"
    u = w.extra.get("u")
    return {"workload": f"{w.name}: {w.nx}x{w.ny}x{w.nz} Q1 hex {w.bc}, {prec}, single reduced-Newton solve",
            "smoother": smoother,
            "grid": [w.nx, w.ny, w.nz], "support": w.bc, "load": w.loads[0], "density": w.density,
            "volume_fraction": w.vf, "levels": w.levels, "rtol": w.rtol, "precision": precision,
            "state_u": (f"seeded smooth field (seed {u[1]}, max |u| = {u[2]})" if u else
                        "equilibrium displacement of K(rho) u = f (library FP64 solve, untimed)"),
            "n_dofs": w.n, "m_elements": w.m,
            "l2": "flushed: a 256 MiB buffer is written between timed steps (outside the step's events)"}


# ------------------------------------------------------------------------------------------------------------
# distributed plumbing
# ------------------------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, device) -> float:
    """The largest of every rank's timed total (the job's time); the value itself with one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, total_ms: float) -> float:
    """Systems per second of the whole job: every rank solves `steps` systems (replicas, weak scaling)."""
    return world * steps / (total_ms / 1e3)


# ------------------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------------------
# roofline helpers
# ------------------------------------------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_hash(precision: str) -> str:
    h = hashlib.sha256()
    for p, marker in KERNEL_SOURCES[precision]:
        with open(p, "rb") as fh:
            txt = fh.read()
        cut = txt.find(marker.encode()) if marker else -1
        h.update(txt if cut < 0 else txt[:cut])
    return h.hexdigest()[:16]


def profiled_traffic(name: str, precision: str):
    """DRAM bytes per launch of the named kernel from the committed ncu summary under profiles/, if it was taken
    on the current kernel source (its `kernel_source_sha` line matches); else None."""
    path = os.path.join(PROFILE_DIR, name)
    try:
        with open(path) as fh:
            txt = fh.read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != kernel_hash(precision):
        return None
    return float(m_tr.group(1))


# ------------------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------------------
REF_DIR = os.path.join(ROOT, "tests", "golden")


def oracle_reference(w, rho, f, u):
    """The oracle's stored reference solution of the workload's reduced system, if one exists and was written for
    these inputs (their sums and norms agree to 1e-12 relative); else (None, reason)."""
    npy = os.path.join(REF_DIR, f"{w.name}_dz_ref.npy")
    meta_path = os.path.join(REF_DIR, f"{w.name}_dz_ref.json")
    if not (os.path.exists(npy) and os.path.exists(meta_path)):
        return None, f"no stored oracle reference for {w.name}"
    with open(meta_path) as fh:
        meta = json.load(fh)
    ramp = np.linspace(1.0, 2.0, u.size)
    mine = {"rho_sum": float(rho.sum()), "rho_norm": float(np.linalg.norm(rho)), "f_norm": float(np.linalg.norm(f)),
            "u_norm": float(np.linalg.norm(u)), "u_ramp": float(u @ ramp)}
    theirs = meta.get("inputs_check", {})
    for k, v in mine.items():
        if k not in theirs or not abs(v - theirs[k]) <= 1e-12 * max(abs(theirs[k]), 1e-300):
            return None, f"stored oracle reference was written for other inputs ({k})"
    return (np.load(npy), meta), None


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1904_06556_gb300 as pkg

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w = synthetic.WORKLOADS[args.workload]
    precision = args.precision
    other = "fp64" if (precision == "mixed" and not args.no_compare) else None

    def t64(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    # ---- inputs (untimed): density, load, the state's displacement, synthetic Newton state ----
    rho = synthetic.density_for(w)
    f_h = synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0])
    f = t64(f_h)
    u_h = synthetic.state_displacement(w)
    uinfo = None
    if u_h is None:
        # the equilibrium of K(rho) u = f by the library's FP64 K solve, to the workload's tolerance
        with pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision="fp64") as G64:
            G64.set_density(t64(rho))
            u, uinfo = G64.minres_solve("K", f, rtol=w.rtol, maxit=2000, check=False)
        if not uinfo["relres"] <= 1e-6:
            raise RuntimeError(f"equilibrium solve of the input state failed: {uinfo}")
        u_h = u.cpu().numpy()
    else:
        u = t64(u_h)
    st_h = synthetic.synthetic_state(w, u_h)
    sd = {k: t64(st_h[k]) for k in ("nu_lo", "nu_up", "rho", "mu_lo", "mu_up")}
    sd["u"] = u
    sd.update({k: float(st_h[k]) for k in ("alpha", "p", "q_lo", "q_up", "V", "rho_lo", "rho_up")})
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > 2 x L2

    def make_grid(prec):
        G = pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision=prec, smoother=args.smoother)
        G.set_density(t64(rho))
        return G

    def make_step(G, last, ph=None):
        def step():
            if ph:
                ph[0].record(stream)
            G.set_state(sd)
            if ph:
                ph[1].record(stream)
            rhs = G.reduced_rhs(f)
            if ph:
                ph[2].record(stream)
            x, info = G.minres_solve("S", rhs, rtol=w.rtol, maxit=1000)
            if ph:
                ph[3].record(stream)
            last["info"] = info
            last["x"] = x
            return x
        return step

    def timed(step, last, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        its = []
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            its.append(last["info"]["iterations"])
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], its

    # ---- the measured precision ----
    G = make_grid(precision)
    last = {}
    ph = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    step = make_step(G, last, ph)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n0 = pkg.kernel_launches()
    step_ms, iters = timed(step, last, args.steps)
    launches = pkg.kernel_launches() - n0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    phases = {"set_state_ms": ph[0].elapsed_time(ph[1]), "rhs_ms": ph[1].elapsed_time(ph[2]),
              "minres_ms": ph[2].elapsed_time(ph[3])}
    x_main = last["x"].detach().cpu().numpy()
    info_main = last["info"]
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    value = whole_job_rate(world, args.steps, total_ms)

    # ---- the same steps again with every fine-level S launch bracketed by CUDA events on its stream
    # (pbm_profile): the roofline's kernel durations. Profiled solves launch eagerly, because an
    # event pair cannot bracket a kernel inside the captured MINRES graph; the kernels are the same.
    G.profile(True)
    G.profile_read("S")
    G.profile_read("K")
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = G.profile_read("S")
    G.profile(False)

    # ---- end to end through the C ABI: pinned host inputs in, solution out, every step ----
    host_in = {k: torch.as_tensor(np.ascontiguousarray(st_h[k] if k != "u" else u_h), dtype=torch.float64)
               .pin_memory() for k in ("u", "nu_lo", "nu_up", "rho", "mu_lo", "mu_up")}
    host_in["f"] = torch.as_tensor(f_h, dtype=torch.float64).pin_memory()
    host_out = torch.empty(w.n + 1, dtype=torch.float64).pin_memory()
    dev_in = {k: torch.empty_like(v, device=dev) for k, v in host_in.items()}
    sd_e2e = {k: dev_in[k] for k in ("u", "nu_lo", "nu_up", "rho", "mu_lo", "mu_up")}
    sd_e2e.update({k: sd[k] for k in ("alpha", "p", "q_lo", "q_up", "V", "rho_lo", "rho_up")})
    h2d = sum(v.numel() * 8 for v in host_in.values())
    d2h = host_out.numel() * 8

    def step_e2e():
        for k, v in host_in.items():
            dev_in[k].copy_(v, non_blocking=True)
        G.set_state(sd_e2e)
        rhs = G.reduced_rhs(dev_in["f"])
        x, _ = G.minres_solve("S", rhs, rtol=w.rtol, maxit=1000)
        host_out.copy_(x, non_blocking=True)

    step_e2e()
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev2[i][0].record(stream)
        step_e2e()
        ev2[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev2)), dev)
    e2e_value = whole_job_rate(world, args.steps, e2e_ms)
    solve = {"minres_iterations": iters[-1], "true_relres": info_main["relres"], "phases_last_step": phases,
             "mixed_outer_steps": info_main["outer"], "fine_chunk": G.info()["fine_chunk"],
             "fp32_tile_K_S": G.info()["fp32_tile"], "fp32_coarse_plans_K_S": G.info()["coarse_plan"],
             "step_ms_min": min(step_ms),
             "step_ms_median": statistics.median(step_ms)}
    if uinfo is not None:
        solve["equilibrium_u_relres"] = uinfo["relres"]
    kapply = k_apply_rates(G, w, rho, dev, flush)
    G.close()

    # ---- the other precision on the same inputs, same protocol (the metric's FP32-mixed vs FP64 comparison) ----
    x_other = None
    if other:
        G2 = make_grid(other)
        last2 = {}
        step2 = make_step(G2, last2)
        for _ in range(args.warmup):
            step2()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms2, its2 = timed(step2, last2, args.steps)
        tot2 = max_over_ranks(float(sum(ms2)), dev)
        x_other = last2["x"].detach().cpu().numpy()
        solve["compare"] = {"precision": other, "systems_per_s": whole_job_rate(world, args.steps, tot2),
                            "ms_per_step": tot2 / args.steps, "minres_iterations": its2[-1],
                            "true_relres": last2["info"]["relres"], "step_ms_median": statistics.median(ms2)}
        solve["speedup_vs_" + other] = (tot2 / args.steps) / (total_ms / args.steps)
        G2.close()

    # ---- error of each solution against the oracle's reference solution (outside every timed region) ----
    ref, why = oracle_reference(w, rho, f_h, u_h)
    if ref is not None:
        dz_ref, meta = ref
        nref = float(np.linalg.norm(dz_ref))
        solve["error_vs_oracle"] = float(np.linalg.norm(x_main - dz_ref) / nref)
        if x_other is not None:
            solve["compare"]["error_vs_oracle"] = float(np.linalg.norm(x_other - dz_ref) / nref)
        solve["oracle_reference"] = {"relres": meta["relres"], "iterations": meta["iterations"],
                                     "solver": meta["solver"]}
    else:
        solve["error_vs_oracle"] = None
        solve["oracle_reference"] = why

    # ---- roofline of the fine-level S kernel ----
    peaks, peak_src = measured_peaks()
    avg_ms = prof["total_ms"] / max(prof["launches"], 1)
    of = "of measured" if peak_src == "measured" else "of fallback"
    if precision == "fp64":
        achieved = prof["flops"] / (prof["total_ms"] / 1e3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_OPS_PEAK / 1e9, "unit": "G FP64 op/s",
                "frac": achieved / (FP64_OPS_PEAK / 1e9),
                "peak_source": "derived: nominal 1.25 TFLOP/s FP64 = 2 FP64 ops/clk/SM x 152 SMs x 2070 MHz",
                "kernel": ("fine-level S operator: k_cols_fine<double, S> (element columns) + k_nodes<double> "
                           "(node sums with the fused residual / Jacobi / dot epilogues), timed as one launch pair")}
        hbm = prof["bytes"] / (prof["total_ms"] / 1e3) / 1e9
        roof["hbm_achieved_gbs"] = hbm
        roof["hbm_frac_" + of.replace(" ", "_")] = hbm / peaks["hbm_gbs"]
    else:
        achieved = prof["bytes"] / (prof["total_ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peak_src} (MEASURED_PEAKS hbm_gbs), {of}",
                "kernel": "fine-level FP32 S operator (single pass, the autotuned plan in fp32_tile_K_S[1]) with its "
                          "fused residual / Jacobi / Chebyshev / dot epilogues, every launch of the solve"}
    roof.update({"launches": prof["launches"], "avg_launch_us": avg_ms * 1e3,
                 "bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                 "ops_per_launch": prof["flops"] / max(prof["launches"], 1)})
    roof["traffic"] = profiled_traffic(f"fine_S_apply_{precision}_{w.name}.md", precision)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded; shapes of the paper's Section 6 examples)",
        "config": workload_desc(w, precision, args.smoother, other),
        "solve": solve,
        "k_apply": kapply,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_budget_s, args.smoother)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_batch(args):
    """Batching workload: 12 design instances of uneven size (3 each of 32x16x16, 48x24x24, 64x32x32 and 96x48x48
    cantilevers, densities U[1e-3, 1] rescaled to mean 0.3, seeds 0..11), each with 4 load cases (end point load,
    distributed end load, top-face traction, torsion couple): 48 reduced-Newton systems. One step = the set-up of every
    system (pbm_set_state), its right-hand side and the solve of all 48 systems, batched (one launch per stage for all
    systems, graph-captured MINRES) or one by one; reports systems per second for both."""
    import torch

    import paper_1904_06556_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precision = args.precision

    def t64(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    grids, states, fs = [], [], []
    for w in synthetic.BATCH_WORKLOADS:
        rho = synthetic.density_for(w)
        with pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision="fp64") as G64:
            G64.set_density(t64(rho))
            for load in w.loads:
                f = t64(synthetic.load_vector(w.nx, w.ny, w.nz, load))
                u, inf = G64.minres_solve("K", f, rtol=w.rtol, maxit=2000, check=False)
                st_h = synthetic.synthetic_state(w, np.zeros(w.n))
                sd = {k: t64(st_h[k]) for k in ("nu_lo", "nu_up", "rho", "mu_lo", "mu_up")}
                sd["u"] = u
                sd.update({k: float(st_h[k]) for k in ("alpha", "p", "q_lo", "q_up", "V", "rho_lo", "rho_up")})
                G = pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision=precision, smoother=args.smoother)
                grids.append(G)
                states.append(sd)
                fs.append(f)
    B = pkg.Batch(grids, "S")
    rtol = synthetic.BATCH_WORKLOADS[0].rtol
    stream = torch.cuda.current_stream()
    last = {}

    def setup():
        rhs = []
        for G, sd, f in zip(grids, states, fs):
            G.set_state(sd)
            rhs.append(G.reduced_rhs(f))
        return rhs

    def step_batched():
        rhs = setup()
        xs, infos = B.minres_solve(rhs, rtol=rtol, maxit=2000)
        last["b"] = infos

    def step_single():
        rhs = setup()
        infos = []
        for G, r in zip(grids, rhs):
            _, inf = G.minres_solve("S", r, rtol=rtol, maxit=2000)
            infos.append(inf)
        last["s"] = infos

    res = {}
    for name, fn in (("batched", step_batched), ("one_by_one", step_single)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = pkg.kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms_per_step": ms, "systems_per_s": len(grids) / (ms / 1e3),
                     "gpu_launches_per_step": (pkg.kernel_launches() - n0) / args.steps}
    ib, i1 = last["b"], last["s"]
    out = {"metric": METRIC + " (batching workload)", "value": res["batched"]["systems_per_s"],
           "unit": "reduced-Newton systems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res["batched"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if precision == "mixed" else "f64",
           "data": "synthetic (seeded; 12 cantilever instances x 4 load cases)",
           "config": {"workload": "batch48: 3 each of 32x16x16, 48x24x24, 64x32x32, 96x48x48 cantilevers, "
                                  "4 load cases each", "systems": len(grids), "precision": precision, "rtol": rtol},
           "batched": res["batched"], "one_by_one": res["one_by_one"],
           "speedup_vs_one_by_one": res["one_by_one"]["ms_per_step"] / res["batched"]["ms_per_step"],
           "iterations_batched": [x["iterations"] for x in ib], "iterations_one_by_one": [x["iterations"] for x in i1],
           "max_relres_batched": max(x["relres"] for x in ib)}
    B.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_ip(args):
    """Interior-point Newton systems (Section 4.1) on the workload's grid: state set-up (coefficients, Galerkin
    hierarchy of S_IP), right-hand side, MG-MINRES to the workload's tolerance and the recovery of the density and
    multiplier increments, at a strictly feasible synthetic point (rho from the density recipe, nu_lo = nu_up = 1,
    alpha = 1, r = s = 1e-2, u the equilibrium displacement). Device-resident inputs, L2 flushed between steps."""
    import torch

    import paper_1904_06556_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synthetic.WORKLOADS[args.workload]

    def t64(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    rho = np.clip(synthetic.density_for(w), 2 * w.rho_lo, 0.99 * w.rho_up)
    f = t64(synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0]))
    with pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision="fp64") as G64:
        G64.set_density(t64(rho))
        u, _ = G64.minres_solve("K", f, rtol=w.rtol, maxit=2000, check=False)
    G = pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision=args.precision, smoother=args.smoother)
    sd = dict(u=u, rho=t64(rho), nu_lo=t64(np.ones(w.m)), nu_up=t64(np.ones(w.m)), alpha=1.0, V=float(rho.sum()),
              rho_lo=w.rho_lo, rho_up=w.rho_up, r=1e-2, s=1e-2)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    last = {}

    def step():
        G.ip_set_state(sd)
        rhs = G.ip_reduced_rhs(f)
        dz, info = G.ip_solve(rhs, rtol=w.rtol, maxit=1000)
        G.ip_recover(dz)
        last["info"] = info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), dev)
    out = {"metric": METRIC + " (interior-point Newton system)", "value": whole_job_rate(world, args.steps, total_ms),
           "unit": "interior-point Newton systems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic (seeded; strictly feasible interior point on the workload's grid)",
           "config": dict(workload_desc(w, args.precision, args.smoother),
                          workload=f"{w.name}: {w.nx}x{w.ny}x{w.nz} Q1 hex {w.bc}, {args.precision}, one "
                                   f"interior-point Newton system (set-up, rhs, MG-MINRES, recovery)"),
           "solve": {"minres_iterations": last["info"]["iterations"], "true_relres": last["info"]["relres"],
                     "outer": last["info"]["outer"]}}
    G.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_doc(args):
    """A complete run of Algorithm DOC (pbm_doc_solve) from the uniform density V/m with the paper's settings
    (q = 1/2, eps_DOC = 1e-3, tau_alpha = eps_DOC / 10, MINRES to 1e-4): total time, DOC and MINRES iterations and
    the final compliance; with --compare-fp64 the other precision too."""
    import torch

    import paper_1904_06556_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synthetic.WORKLOADS[args.workload]
    f = torch.as_tensor(synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0]), dtype=torch.float64, device=dev)

    def one_run(precision):
        with pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision=precision, smoother=args.smoother) as G:
            rho = torch.full((w.m,), w.V / w.m, dtype=torch.float64, device=dev)
            u = torch.zeros(w.n, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = G.doc_solve(rho, f, u, w.V, w.rho_lo, w.rho_up, check=False, eps_doc=1e-3, eps_mr=1e-4)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, info

    secs, info = one_run(args.precision)
    out = {"metric": METRIC + " (complete DOC run)", "value": secs, "unit": "s per DOC run", "n_gpus": world,
           "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if args.precision == "mixed" else "f64",
           "data": "synthetic (seeded; the paper's cantilever example, Section 6)",
           "config": dict(workload_desc(w, args.precision, args.smoother),
                          workload=f"{w.name}: {w.nx}x{w.ny}x{w.nz} Q1 hex {w.bc}, {args.precision}, complete DOC "
                                   f"run (q 1/2, eps_DOC 1e-3, MINRES 1e-4)"),
           "doc": info}
    if args.compare_fp64:
        s2, i2 = one_run("fp64" if args.precision == "mixed" else "mixed")
        out["other_precision"] = {"seconds": s2, "iterations": i2["iterations"], "minres": i2["minres"],
                                  "compliance": i2["compliance"]}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_pbm(args):
    """A complete PBM run (Algorithm 1, pbm_solve) from the paper's initial point on the workload's grid: the
    large full-PBM workload (256 x 128 x 128 cantilever, distributed end load, vf 0.15, 7 levels) or any other
    grid. Reports the total time, the outer / Newton / MINRES counts, the compliance and the fine-level
    K(rho) x roofline at that size; with --compare-fp64 the same run with the FP64 path and the relative
    difference of the compliances. Rank 0 only (replicas otherwise do the same run)."""
    import torch

    import paper_1904_06556_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synthetic.WORKLOADS[args.workload]
    f = torch.as_tensor(synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0]), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def one_run(precision):
        with pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision=precision, smoother=args.smoother) as G:
            st = G.initial_state(w.n, w.m, w.V, w.rho_lo, w.rho_up, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = G.pbm_solve(st, f, check=False)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            rho = st["rho"]
            kap = k_apply_rates(G, w, rho.cpu().numpy(), dev, flush) if precision == args.precision else None
        return secs, info, kap, float(rho.sum().item())

    secs, info, kap, vol = one_run(args.precision)
    peaks, peak_src = measured_peaks()
    out = {"metric": METRIC + " (full PBM run)", "value": secs, "unit": "s per PBM run", "n_gpus": world,
           "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if args.precision == "mixed" else "f64",
           "data": "synthetic (seeded; the paper's cantilever example, Section 6)",
           "config": dict(workload_desc(w, args.precision, args.smoother),
                          workload=f"{w.name}: {w.nx}x{w.ny}x{w.nz} Q1 hex {w.bc}, {args.precision}, complete PBM "
                                   f"run from the paper's initial point (eps_pbm 1e-5)"),
           "pbm": {k: info[k] for k in ("rc", "status", "outer", "newton", "minres", "gap_ratio", "compliance",
                                        "volume", "eps_mr")},
           "volume_fraction_final": vol / w.m,
           "k_apply": kap,
           "k_apply_roofline_fp32": {"bound": "hbm", "achieved": kap["fp32"]["gbs_flushed"],
                                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                     "frac": kap["fp32"]["gbs_flushed"] / peaks["hbm_gbs"],
                                     "peak_source": peak_src}}
    if args.compare_fp64:
        s64, i64, _, _ = one_run("fp64" if args.precision == "mixed" else "mixed")
        out["other_precision"] = {"seconds": s64, "outer": i64["outer"], "newton": i64["newton"],
                                  "minres": i64["minres"], "compliance": i64["compliance"],
                                  "compliance_rel_diff": abs(info["compliance"] - i64["compliance"]) /
                                  abs(i64["compliance"])}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_plans(args):
    """Times every tile plan of the single-pass FP32 operator (pbm_set_fp32_plan) on the workload's grid, K and S
    with the apply epilogue: median of 20 launches with the L2 flushed before each (CUDA events). Prints one JSON
    line per plan and operator."""
    import torch

    import paper_1904_06556_gb300 as pkg

    _, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synthetic.WORKLOADS[args.workload]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    G = pkg.Grid(w.nx, w.ny, w.nz, w.levels, w.bc, precision="mixed")
    G.set_density(torch.as_tensor(synthetic.density_for(w), dtype=torch.float64, device=dev))
    G.vcycle("K", torch.zeros(w.n, dtype=torch.float64, device=dev))
    x = torch.randn(w.n + 1, dtype=torch.float32, device=dev)

    def med_us(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(20):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return statistics.median(ts)

    st_h = synthetic.synthetic_state(w, np.zeros(w.n))
    sd = {k: torch.as_tensor(st_h[k], dtype=torch.float64, device=dev) for k in ("nu_lo", "nu_up", "rho", "mu_lo",
                                                                                   "mu_up")}
    sd["u"] = 1e-2 * torch.randn(w.n, dtype=torch.float64, device=dev)
    sd.update({k: float(st_h[k]) for k in ("alpha", "p", "q_lo", "q_up", "V", "rho_lo", "rho_up")})
    peaks, _ = measured_peaks()
    for op, nv, byt in (("K", w.n, (2 * w.n + w.m) * 4), ("S", w.n + 1, (3 * w.n + 2 * w.m) * 4)):
        if op == "S":
            G.set_state(sd)
        for plan in range(pkg.fp32_plan_count()):
            G.set_fp32_plan(op, plan)
            us = med_us(lambda: G.apply_fine_f32(op, "apply", x[:nv]))
            tile = G.info()["fp32_tile"][0 if op == "K" else 1]
            print(json.dumps({"workload": w.name, "op": op, "plan": plan, "tile_TX_TY_DZ_threads": tile[:4],
                              "us_flushed": us, "gbs": byt / us / 1e3, "frac_of_hbm": byt / us / 1e3 /
                              peaks["hbm_gbs"]}), flush=True)
    G.close()


def k_apply_rates(G, w, rho, dev, flush):
    """Standalone fine-level K(rho) x in FP64 and FP32 at the workload size: algorithmic GB/s = (2n + m) b /
    kernel time, with the L2 flushed before every launch and warm (back to back)."""
    import torch
    n, m = w.n, w.m
    x64 = torch.randn(n, dtype=torch.float64, device=dev)
    w64 = torch.as_tensor(rho, dtype=torch.float64, device=dev)
    y64 = torch.empty_like(x64)
    x32, w32 = x64.float(), w64.float()
    y32 = torch.empty_like(x32)
    res = {}
    for name, fn, b in (("fp64", lambda: G.apply_K(x64, w64, out=y64), 8),
                        ("fp32", lambda: G.apply_K_f32(x32, w32, out=y32), 4)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        cold = []
        for _ in range(10):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            cold.append(e0.elapsed_time(e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(50):
            fn()
        e1.record()
        torch.cuda.synchronize()
        warm = e0.elapsed_time(e1) / 50
        byt = (2 * n + m) * b
        cold_ms = statistics.median(cold)
        res[name] = {"us_flushed": cold_ms * 1e3, "gbs_flushed": byt / (cold_ms / 1e3) / 1e9,
                     "us_warm": warm * 1e3, "gbs_warm": byt / (warm / 1e3) / 1e9, "bytes": byt}
    return res


# ------------------------------------------------------------------------------------------------------------
# the CPU oracle (the cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------------------------
def oracle_inputs(w):
    from oracle import fem, pbm, solvers
    g = fem.Grid(w.nx, w.ny, w.nz, w.bc)
    rho = synthetic.density_for(w)
    f = synthetic.load_vector(w.nx, w.ny, w.nz, w.loads[0])
    u = synthetic.state_displacement(w)
    if u is None:
        K = fem.assemble_K(g, rho, fem.element_stiffness(w.E, w.nu))
        h = solvers.Hierarchy(g, K, w.levels, has_alpha=False)
        u = solvers.minres(lambda v: K @ v, f, h.vcycle, rtol=1e-12, maxit=2000).x
    d = synthetic.synthetic_state(w, u)
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    return pb, pbm.State.from_dict(d)


def oracle_step(w, pb, st, smoother="jacobi", levels=None, maxit=1000, rtol=None):
    """One reduced Newton system by the oracle: coefficients, S in CSR, Galerkin hierarchy, rhs, MG-MINRES.
    Returns (MINRES result, set-up seconds, solve seconds)."""
    from oracle import pbm, solvers
    t0 = time.perf_counter()
    cf = pbm.coeffs(pb, st)
    S = pbm.assemble_S(pb, st, cf)
    rhs = pbm.rhs_closed(pb, st, cf)
    h = solvers.Hierarchy(pb.grid, S, levels or w.levels, has_alpha=True, smoother=smoother)
    t1 = time.perf_counter()
    r = solvers.minres(lambda v: S @ v, rhs, h.vcycle, rtol=rtol or w.rtol, maxit=maxit)
    return r, t1 - t0, time.perf_counter() - t1


# workloads whose complete oracle system takes more than a few seconds are sampled: an x-slab of the same grid,
# densities and state (every element's set-up and every MINRES iteration cost the same per element), timed for its
# set-up and a few MG-MINRES iterations, scaled to the full element count and to the oracle's own iteration count
SLAB_NX = {"bridge128": 16, "cant256": 16}


def _slab(w, nx_s):
    """The x-slab [0, nx_s] of workload w: its grid, densities, state displacement and load, as an oracle problem."""
    from oracle import fem, pbm
    rho = synthetic.density_for(w).reshape(w.nz, w.ny, w.nx)[:, :, :nx_s].ravel()
    u_full = synthetic.state_displacement(w)
    if u_full is None:
        u_full = synthetic.smooth_displacement(w.nx, w.ny, w.nz, 5, 1.0)
    u = u_full.reshape(w.nz + 1, w.ny + 1, w.nx + 1, 3)[:, :, :nx_s + 1, :].ravel().copy()
    g = fem.Grid(nx_s, w.ny, w.nz, w.bc)
    u[g.fixed_dofs()] = 0.0
    f = synthetic.load_vector(nx_s, w.ny, w.nz, w.loads[0])
    m = g.m
    d = dict(u=u, alpha=1.0, nu_lo=np.ones(m), nu_up=np.ones(m), rho=rho, mu_lo=np.ones(m), mu_up=np.ones(m),
             p=1.0, q_lo=1.0, q_up=1.0, V=w.vf * m, rho_lo=w.rho_lo, rho_up=w.rho_up)
    return pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"]), pbm.State.from_dict(d)


def oracle_sample_seconds(w, smoother, ctx):
    """Seconds of one complete reduced Newton system of workload w by the oracle, measured on a bounded sample.
    ctx caches the sample's inputs across calls. Returns (seconds, description of the sample)."""
    nx_s = SLAB_NX.get(w.name)
    if nx_s is None:
        if "full" not in ctx:
            ctx["full"] = oracle_inputs(w)
        pb, st = ctx["full"]
        r, ts, tm = oracle_step(w, pb, st, smoother)
        return ts + tm, (f"the complete system (coefficients, CSR S, Galerkin hierarchy, rhs, MG-MINRES to "
                         f"{w.rtol:g}: {r.iters} iterations)")
    if "slab" not in ctx:
        ctx["slab"] = _slab(w, nx_s)
        meta_path = os.path.join(REF_DIR, f"{w.name}_dz_ref.json")
        iters = None
        if os.path.exists(meta_path):
            with open(meta_path) as fh:
                iters = json.load(fh).get("iterations_to_1e-8")
        ctx["iters"] = iters or 40
    pb, st = ctx["slab"]
    k = 3
    levels = min(w.levels, int(np.log2(nx_s)) + 1)
    r, ts, tm = oracle_step(w, pb, st, smoother, levels=levels, maxit=k, rtol=1e-30)
    scale = w.m / pb.grid.m
    per_it = tm / max(r.iters, 1)
    secs = scale * (ts + ctx["iters"] * per_it)
    return secs, (f"x-slab {nx_s}x{w.ny}x{w.nz} (1/{scale:g} of the elements) of the same system: set-up "
                  f"(coefficients, CSR S, {levels}-level Galerkin hierarchy, rhs) and {r.iters} MG-MINRES "
                  f"iterations timed, scaled by {scale:g} to the full element count and to the "
                  f"{ctx['iters']} iterations the oracle needs to {w.rtol:g} on the full system")


def oracle_spmv(w, ctx):
    """The oracle's CSR product K(rho) x on the sample's grid (scipy, single-threaded): seconds per product scaled
    to the full element count, and its rate in algorithmic bytes ((2n + m) 8 per product, the FP64 K(w) x bytes)."""
    from oracle import fem
    pb, st = ctx.get("slab") or ctx["full"]
    g = pb.grid
    K = fem.assemble_K(g, st.rho, fem.element_stiffness(w.E, w.nu))
    x = np.random.default_rng(0).standard_normal(g.n)
    y = K @ x
    ts = []
    for _ in range(10):
        t0 = time.perf_counter()
        y = K @ x
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    scale = w.m / g.m
    return {"ms_per_product_full_size": 1e3 * t * scale, "gbs_algorithmic": (2 * g.n + g.m) * 8 / t / 1e9,
            "csr_nonzeros": int(K.nnz), "threads": 1,
            "sample": f"K(rho) x on the {g.nx}x{g.ny}x{g.nz} sample grid, median of 10, scaled by {scale:g}"}


def cpu_baseline(w, budget_s, smoother="jacobi"):
    ctx = {}
    times, desc = [], ""
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        secs, desc = oracle_sample_seconds(w, smoother, ctx)
        times.append(secs)
        if time.perf_counter() - t_all + (time.perf_counter() - t0) > budget_s or len(times) >= 5:
            break
    tm = statistics.median(times)
    spmv = oracle_spmv(w, ctx)
    return {"value": 1.0 / tm, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "spmv_K": spmv,
            "blas_threads": int(os.environ.get("OPENBLAS_NUM_THREADS", "1")),
            "sample": (f"{len(times)} sample(s): {desc}; median {tm:.2f} s per system; BLAS/OpenMP threads = "
                       f"{os.environ.get('OPENBLAS_NUM_THREADS')} of {os.cpu_count()} host cores (dense coarsest "
                       f"factorisation), scipy sparse products single-threaded")}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = synthetic.WORKLOADS[args.workload]
    ctx = {}
    budget = args.cpu_budget_s * 6
    t_start = time.perf_counter()
    desc = ""
    for _ in range(min(args.warmup, 1)):
        _, desc = oracle_sample_seconds(w, args.smoother, ctx)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        secs, desc = oracle_sample_seconds(w, args.smoother, ctx)
        times.append(secs)
        if time.perf_counter() - t_start + (time.perf_counter() - t0) > budget:
            break
    total = sum(times)
    value = len(times) / total
    other = "fp64" if (args.precision == "mixed" and not args.no_compare) else None
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": len(times), "steps_requested": args.steps, "warmup": min(args.warmup, 1),
           "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
           "config": workload_desc(w, args.precision, args.smoother, other),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "blas_threads": int(os.environ.get("OPENBLAS_NUM_THREADS", "1")),
                            "sample": f"every step: {desc}"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bridge128",
                    choices=["cant64", "bridge128", "cant32", "cant16", "cant256", "batch48"])
    ap.add_argument("--pbm", action="store_true", help="time one complete PBM run (Algorithm 1) on the workload")
    ap.add_argument("--ip", action="store_true", help="time interior-point Newton systems (Section 4.1)")
    ap.add_argument("--doc", action="store_true", help="time one complete run of Algorithm DOC")
    ap.add_argument("--compare-fp64", action="store_true", help="with --pbm: also run the other precision")
    ap.add_argument("--fp32-plans", action="store_true",
                    help="time every tile plan of the FP32 fine operator on the workload's grid")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true",
                    help="with --precision mixed: skip the FP64 solve of the same system")
    ap.add_argument("--smoother", default="chebyshev", choices=["jacobi", "chebyshev", "gauss_seidel"],
                    help="V-cycle smoothing: Chebyshev acceleration of Jacobi (default; fewer MINRES iterations "
                         "for the same operator applications) or damped Jacobi")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=30.0)
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("--steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch48":
        run_batch(args)
    elif args.pbm:
        run_pbm(args)
    elif args.ip:
        run_ip(args)
    elif args.doc:
        run_doc(args)
    elif args.fp32_plans:
        run_plans(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
