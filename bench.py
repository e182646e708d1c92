#!/usr/bin/env python
"""Throughput of the FLO-SIC step: orbital SIC solves per second at 128^3.

One step is the whole hot path on one batch: Fermi-Loewdin orbitals, one
Poisson solve per orbital, LSDA energies and the averaged SIC potential,
then the adjoint (dE_SIC/dpsi and FOD gradients).  Workload: 128^3 grid,
h = 0.2 bohr, 32 + 32 orbitals on 16 seeded atoms (synthetic Gaussian
s/p orbitals, seeded FODs), forward + adjoint.  value = orbitals / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--precision mixed|fp64] [--solver kron|pcg|aar]
                  [--workload 128|192|uneven|fodopt|hamiltonian]
                  [--no-cpu-baseline] [--no-e2e] [--no-fp64] [--no-pcg]

The Poisson solves run in mixed precision with the Kronecker-product inner
solver by default (the exact float32 inverse of the discrete operator inside
the float-float refinement, to ||r|| <= 1e-10 ||b||); the line also carries
the same step with multigrid-preconditioned CG (pcg_path) and with the plain
float64 path (fp64_path).

Under torchrun (N > 1) the orbitals of the one 128^3 system are split over
the ranks by default (--shard orbitals: every rank builds all FLOs, solves
and scores its own orbitals, and E_SIC, V_avg, the energies and gradients
are summed over ranks with NCCL; strong scaling, value = the system's
orbitals / max time); --shard systems gives every rank its own independent
system instead (weak scaling, value = all orbitals / max time).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "orbital SIC solves/s at 128^3, mixed vs FP64 at 1e-6 Ha; HBM % of peak"
WORKLOAD = "128^3 grid h=0.2 bohr, 32+32 orbitals on 16 atoms, FLO build + 64 Poisson solves + LSDA/E_SIC/V_avg + adjoint"
METRIC_192 = "orbital SIC solves/s at 192^3 (120+120 orbitals), mixed precision; HBM % of peak"
WORKLOAD_192 = ("192^3 grid h=0.15 bohr, 120+120 orbitals on 60 atoms, FLO build (tensor-core overlap) + 240 "
                "Poisson solves + LSDA/E_SIC/V_avg + adjoint")
CG_TOL = 1e-10
# Plain-CG iterations the oracle needs per orbital of this workload to reach
# ||r|| <= 1e-10 ||b|| (measured once on orbital 0 of spin 0); used to scale the
# oracle's timed sample of iterations up to whole solves.
ORACLE_CG_ITERS_128 = 687


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--preconditioner", default="mg", choices=["mg", "none"])
    p.add_argument("--solver", default="kron", choices=["pcg", "aar", "kron"],
                   help="float32 inner solver of the mixed path: CG, Alternating Anderson-Richardson, "
                        "or the Kronecker-product eigen-solver")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-pcg", action="store_true", help="skip the multigrid-PCG comparison line")
    p.add_argument("--shard", default="orbitals", choices=["orbitals", "systems"],
                   help="N > 1: split the orbitals of one system over the ranks (strong scaling; every rank "
                        "builds all FLOs, solves and scores its own orbitals, sums over ranks) or give every "
                        "rank its own system (weak scaling)")
    p.add_argument("--no-tensor-core-transforms", action="store_true",
                   help="Kronecker solver: keep every 1-D transform on the CUDA cores")
    p.add_argument("--no-extra-workloads", action="store_true",
                   help="skip the uneven-batch and 192^3 lines added to the default line")
    p.add_argument("--workload", default="128", choices=["128", "192", "uneven", "fodopt", "hamiltonian"],
                   help="128: the 128^3 forward+adjoint step (default); 192: the same step at 192^3 with "
                        "120+120 orbitals; uneven: 64 systems of "
                        "48^3..128^3 grids and 2..40 orbitals, forward step; fodopt: FIRE FOD relaxation "
                        "steps at 128^3; hamiltonian: SC_AvgSIC Hamiltonian apply at 128^3")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax = max(smax, float(f[1]))
            except ValueError:
                continue
            for k, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle, timed on the host cores on a bounded sample of the workload
# ---------------------------------------------------------------------------
# CG iterations of the two timed Poisson samples; their difference gives the
# oracle's cost per iteration without its per-call set-up (moments, boundary
# values), so short samples do not inflate the extrapolation.
ORACLE_SAMPLE_ITERS = (4, 16)


def oracle_sample(system):
    """Times the FP64 oracle on a bounded sample of one step and extrapolates
    it to solves/s.  The cpu_baseline leg and the reference arm both call this
    one definition.  Measured in full: both spins' FLO build, the LSDA/energy
    pass and the adjoint.  Sampled: the Poisson solves of `cores` orbitals at
    once (OpenMP over orbitals), timed at two iteration counts; the per-
    iteration cost (difference quotient) and the per-call set-up (the
    intercept) are scaled to ORACLE_CG_ITERS_128 iterations and to all
    orbitals, in waves of `cores`."""
    import oracle
    oracle.build_library()
    cores = oracle.max_threads()
    s = system
    nsp = len(s.norb)
    norb = sum(s.norb)
    t0 = time.perf_counter()
    blocks = [oracle.build_flos(s.psi[k], s.fods[k], s.grid) for k in range(nsp)]
    t_build = time.perf_counter() - t0
    rho = np.concatenate([b["phi"] ** 2 for b in blocks])[:cores]
    it_lo, it_hi = ORACLE_SAMPLE_ITERS
    t0 = time.perf_counter()
    oracle.poisson(rho, s.grid, tol=1e-300, max_iter=it_lo)
    t_lo = time.perf_counter() - t0
    t0 = time.perf_counter()
    V, _ = oracle.poisson(rho, s.grid, tol=1e-300, max_iter=it_hi)
    t_hi = time.perf_counter() - t0
    per_it = max(t_hi - t_lo, 1e-9) / (it_hi - it_lo)
    setup = max(t_lo - it_lo * per_it, 0.0)
    # energies and adjoint on the (partly solved) potentials: same work as a full step
    t0 = time.perf_counter()
    fwd = dict(blocks=[], E_sic=0.0)
    for k, b in enumerate(blocks):
        Vk = np.resize(V, b["phi"].shape)
        eps, vxc = oracle.lsda_pol(b["phi"] ** 2)
        b.update(rho=b["phi"] ** 2, V=Vk, eps=eps, vxc=vxc, psi=s.psi[k], fods=s.fods[k])
        fwd["blocks"].append(b)
    t_en = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.sic_backward(fwd, s.grid)
    t_bw = time.perf_counter() - t0
    waves = -(-norb // cores)
    t_wave = setup + ORACLE_CG_ITERS_128 * per_it
    t_full = t_build + waves * t_wave + t_en + t_bw
    elapsed = t_build + t_lo + t_hi + t_en + t_bw
    desc = ("measured in full: FLO build of both spins, LSDA/energies, adjoint; Poisson: %d orbitals at once timed "
            "at %d and %d plain-CG iterations, per-iteration cost and set-up scaled to %d orbitals x %d iterations "
            "(the oracle's own count to 1e-10 on this workload)"
            % (cores, it_lo, it_hi, norb, ORACLE_CG_ITERS_128))
    return dict(value=norb / t_full, unit="solves/s", cores=cores, kind="oracle", sample=desc, extrapolated=True,
                sample_seconds=round(elapsed, 2), extrapolated_step_s=round(t_full, 1),
                measured_s={"flo_build": round(t_build, 3), "poisson_%d_iters" % it_lo: round(t_lo, 3),
                            "poisson_%d_iters" % it_hi: round(t_hi, 3), "energies": round(t_en, 3),
                            "adjoint": round(t_bw, 3)},
                cg_iters_per_solve=ORACLE_CG_ITERS_128)


def run_reference(args):
    """The reference arm: the oracle as it stands on the host cores, one
    bounded sample (oracle_sample, the same definition as the cpu_baseline
    leg) per step; value = the mean of the timed steps' extrapolated
    throughput.  Under torchrun only rank 0 runs and prints."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2108_01186_gb300 import synth
    s = synth.make_config(3)
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        r = oracle_sample(s)
        if k >= args.warmup:
            vals.append(r["value"])
            secs.append(r["sample_seconds"])
    v = statistics.mean(vals)
    cb = dict(r)
    cb["value"] = v
    cb["value_spread"] = [min(vals), max(vals)]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 64 / v,
            "ms_per_step_is": "extrapolated full step (each timed step ran one bounded sample, mean %.1f s)"
                              % statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "system": "FP64 CPU oracle, host cores"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------
def traffic_for(kernel_src):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if d.get("source_sha") != sha:
        return None
    return d.get("traffic_bytes_per_launch_scaled")


def kron_tc_traffic(n_orb):
    """DRAM bytes of the six tensor-core transform passes of one solve, from
    the committed ncu summary (scaled by orbitals), while kron_tc.cu is the
    source the capture was taken on."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "kron_tc_traffic.json")))
        src = os.path.join(ROOT, "paper_2108_01186_gb300", "csrc", "kron_tc.cu")
        if d.get("source_sha") != hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]:
            return None
        return int(d["traffic_bytes_per_solve"] * n_orb / d["orbitals"])
    except (OSError, ValueError, KeyError):
        return None


def step_with(ctx, psi, fods, gE):
    """One forward + adjoint step through the public API."""
    phi, _, _ = ctx.build_flos(psi, fods, want_matrices=False)
    V, iters, conv = ctx.orbital_poisson(phi)
    E, Vavg, U, Exc = ctx.sic_energy_potential(psi, phi, V, 1.0)
    dpsi, dfod = ctx.sic_backward(psi, fods, phi, V, gE)
    return E, Vavg, dpsi, dfod, iters


def step_outputs(ctx, psi, fods):
    phi, _, _ = ctx.build_flos(psi, fods, want_matrices=False)
    V, _, _ = ctx.orbital_poisson(phi)
    return phi, V


def run_gpu(args):
    import torch
    from paper_2108_01186_gb300 import dist as D
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D.init("nccl")
    from paper_2108_01186_gb300 import build, synth
    from paper_2108_01186_gb300.flosic import Context

    build.build()
    sharded = world > 1 and args.shard == "orbitals"
    seed_rank = 0 if sharded else rank   # sharded: one system split over the ranks; else one per rank
    if args.workload == "192":   # the largest workload: 192^3, h=0.15, 120+120 orbitals on 60 atoms
        s = synth.make_system(192, 0.15, 60, [120, 120], seed=4000 + seed_rank)
        workload = WORKLOAD_192
    else:
        s = synth.make_system(128, 0.2, 16, [32, 32], seed=3000 + seed_rank)
        workload = WORKLOAD
    norb = sum(s.norb)
    prec = 1 if args.precision == "mixed" else 0
    pc = 1 if args.preconditioner == "mg" else 0
    solver = {"pcg": 0, "aar": 1, "kron": 2}[args.solver]
    ctx = Context([s], precision=prec, cg_tol=CG_TOL, preconditioner=pc, solver=solver,
                  kron_tensor_cores=0 if args.no_tensor_core_transforms else 1)
    paths = ctx.block_paths()
    if args.no_tensor_core_transforms:
        transforms_desc = "cuda cores"
    else:   # the autotuner's pick per block shape (tensor cores or CUDA cores, timed at context creation)
        ntc = sum(p["tensor_core_transforms"] for p in paths)
        transforms_desc = ("tensor cores (autotuned)" if ntc == len(paths) else
                           "cuda cores (autotuned)" if ntc == 0 else "mixed (autotuned, %d of %d blocks on tensor cores)"
                           % (ntc, len(paths)))
    shard_step = D.OrbitalShardedStep(ctx) if sharded else None
    units = world * norb if not sharded else norb   # orbitals the whole job processes per step
    dev = torch.device("cuda", local)
    psi_h = torch.from_numpy(np.concatenate([p.ravel() for p in s.psi])).pin_memory()
    fods_h = torch.from_numpy(np.concatenate([f.ravel() for f in s.fods])).pin_memory()
    psi = psi_h.to(dev)
    fods = fods_h.to(dev)
    gE = torch.ones(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step(psi, fods):
        if shard_step is None:
            return step_with(ctx, psi, fods, gE)
        out = shard_step.forward(psi, fods, 1.0)
        dpsi, dfod = shard_step.backward(psi, fods, out["phi"], out["V"], gE)
        return out["E_sic"], out["V_avg"], dpsi, dfod, out["iters"]

    def barrier():
        D.barrier(torch.cuda.synchronize)

    for _ in range(args.warmup):
        step(psi, fods)
    barrier()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    ctx.profile_read_overlap(reset=True)
    clk = ClockSampler(local)
    clk.start()
    iters_sum = np.zeros(norb)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        E, Vavg, dpsi, dfod, iters = step(psi, fods)
        iters_sum += iters.cpu().numpy()
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read(reset=True)
    prof_ov = ctx.profile_read_overlap(reset=True)
    ctx.profile(False)
    ms = D.max_over_ranks(ms, dev)
    ms_step = ms / args.steps
    value = units / (ms_step / 1e3)

    # roofline of the dominant kernel (the PCG stencil apply): algorithmic
    # bytes counted on the device per active orbital and launch (read z,
    # p_old, q_old; write p, q -- 20 B/point in float32, 12 B on a solve's
    # first iteration)
    alg_bytes = prof["kernel_bytes"]
    launches = max(prof["kernel_launches"], 1)
    achieved = alg_bytes / (prof["kernel_ms"] / 1e3) / 1e9 if prof["kernel_ms"] > 0 else 0.0
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        peak, peak_src = 6800.0, "fallback"
    kname = "k_apply12_tma<float>" if prec == 1 else "k_apply12_tma<double>"
    if solver == 1:
        kname = "k_residual12_aar<float>"
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": (traffic_for(os.path.join(ROOT, "paper_2108_01186_gb300", "csrc", "stencil.cu"))
                        if args.workload == "128" and solver == 0 else None),
            "alg_bytes_per_launch": alg_bytes / launches,
            "avg_launch_ms": prof["kernel_ms"] / launches, "launches": prof["kernel_launches"],
            "share_of_step": round(prof["kernel_ms"] / ms, 4)}
    if solver == 2:
        # the Kronecker solver's six transform passes per solve (timed by the
        # library around each inner solve; algorithmic flops 2 (n_s^2 + n_a^2)
        # per line and pass counted on the device)
        n_local = sum(shard_step.mask) if shard_step is not None else norb   # orbitals this rank solves
        alg_bytes = 6 * 8 * n_local * s.G          # per solve: every pass reads and writes 4 B per point
        solve_ms = prof["kernel_ms"] / launches
        flops_solve = prof["kernel_bytes"] / launches
        gbs = alg_bytes / (solve_ms / 1e3) / 1e9 if solve_ms > 0 else 0.0
        if not args.no_tensor_core_transforms:
            # tensor-core transforms: HBM-bound (one read and one write of the
            # float32 field per pass); the tensor pipe executes the six split
            # products of every half-size transform
            try:
                pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                tcp, tcs = float(pk["bf16_tflops"]), "measured"
            except (OSError, ValueError, KeyError):
                tcp, tcs = 1900.0, "fallback"
            roof = {"bound": "hbm", "kernel": "k_kron_tc (6 passes per solve; tcgen05, split bf16)",
                    "achieved": round(gbs, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                    "frac": round(gbs / peak, 4),
                    "traffic": (kron_tc_traffic(n_local) if args.workload == "128" else None),
                    "traffic_per": "solve (6 launches)", "alg_bytes_per_solve": alg_bytes,
                    "avg_solve_ms": solve_ms, "launches": prof["kernel_launches"],
                    "share_of_step": round(prof["kernel_ms"] / ms, 4),
                    "tensor_pipe": {"executed_tflops": round(6 * flops_solve / (solve_ms / 1e3) / 1e12, 2)
                                    if solve_ms > 0 else 0.0,
                                    "peak": tcp, "peak_source": tcs,
                                    "frac": round(6 * flops_solve / (solve_ms / 1e3) / 1e12 / tcp, 4)
                                    if solve_ms > 0 else 0.0}}
        else:
            # CUDA-core transforms: float32 FMA-bound dense 1-D products; peak =
            # the device's SMs x 128 FP32 lanes x 2 flops x its maximum SM clock
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            fmax = (clocks or {}).get("sm_max_mhz") or 2070.0
            fp32_peak = sms * 128 * 2 * fmax * 1e6 / 1e12
            tfl = flops_solve / (solve_ms / 1e3) / 1e12 if solve_ms > 0 else 0.0
            roof = {"bound": "alu", "kernel": "k_kron_pass (6 passes per solve)", "achieved": round(tfl, 2),
                    "peak": round(fp32_peak, 1),
                    "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (sms, fmax),
                    "unit": "TFLOP/s", "frac": round(tfl / fp32_peak, 4), "traffic": None,
                    "alg_bytes_per_solve": alg_bytes, "hbm_achieved_gbs": round(gbs, 1),
                    "alg_flops_per_solve": flops_solve, "avg_solve_ms": solve_ms,
                    "launches": prof["kernel_launches"], "share_of_step": round(prof["kernel_ms"] / ms, 4)}
    # the overlap Gram on the tensor cores (mixed path): algorithmic flops
    # 2 N^2 G per spin block against the measured dense bf16 peak, and its
    # float64 reads of psi (8 N G bytes per block) against the HBM peak
    roof_ov = None
    if prof_ov["kernel_launches"] > 0 and prof_ov["kernel_ms"] > 0:
        try:
            pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            tc_peak, tc_src = float(pk["bf16_tflops"]), "measured"
        except (OSError, ValueError, KeyError):
            tc_peak, tc_src = 1900.0, "fallback"
        sec = prof_ov["kernel_ms"] / 1e3
        tflops = prof_ov["flops"] / sec / 1e12
        ov_bytes = prof_ov["kernel_launches"] * sum(8.0 * n * s.G for n in s.norb)
        roof_ov = {"bound": "latency", "kernel": "k_gram_async (split-BF16 tcgen05)",
                   "achieved": round(tflops, 3), "peak": tc_peak, "peak_source": tc_src, "unit": "TFLOP/s",
                   "frac": round(tflops / tc_peak, 5),
                   "hbm_achieved_gbs": round(ov_bytes / sec / 1e9, 1),
                   "hbm_frac": round(ov_bytes / sec / 1e9 / peak, 4),
                   "avg_launch_ms": prof_ov["kernel_ms"] / prof_ov["kernel_launches"],
                   "launches": prof_ov["kernel_launches"]}

    # end to end through the public API with host buffers: flosic_step_host
    # (host arrays in, host arrays out, the library's own copies); two host
    # input sets alternate, so every step copies its inputs, and each call
    # hands the library the next step's inputs, which it copies while this
    # step computes and whose FLO build and Poisson solve it starts while
    # this step's outputs travel to the host (the last call hands none)
    e2e = None
    if not args.no_e2e and shard_step is None:
        psi_h2 = psi_h.clone().pin_memory()
        fods_h2 = fods_h.clone().pin_memory()
        ins = [(psi_h, fods_h), (psi_h2, fods_h2)]
        pin = lambda n, dt=torch.float64: torch.empty(n, dtype=dt).pin_memory()
        o_E, o_U, o_X = pin(ctx.nsys), pin(ctx.norb), pin(ctx.norb)
        o_V, o_dp, o_df, o_cv = pin(ctx.vavg_elems), pin(ctx.orb_elems), pin(3 * ctx.norb), pin(ctx.norb, torch.int32)
        ctx.step_host(psi_h, fods_h, 1.0, 1.0, o_E, o_U, o_X, o_V, o_dp, o_df, o_cv)   # untimed: buffers
        ke = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for k in range(ke):
            nx = ins[(k + 1) % 2] if k + 1 < ke else (None, None)
            ctx.step_host(ins[k % 2][0], ins[k % 2][1], 1.0, 1.0, o_E, o_U, o_X, o_V, o_dp, o_df, o_cv,
                          psi_next=nx[0], fods_next=nx[1])
        barrier()
        te = D.max_over_ranks((time.perf_counter() - t0) / ke, dev)
        e2e = {"value": units / te, "unit": "solves/s", "api": "flosic_step_host (host arrays in and out)",
               "steps": ke, "ms_per_step": 1e3 * te,
               "overlap": "each step's input copy runs during the previous step (the first inside the timed "
                          "region); each step's FLO build and Poisson solve run while the previous step's outputs "
                          "are copied to the host",
               "h2d_bytes_per_step": int(psi_h.numel() * 8 + fods_h.numel() * 8),
               "d2h_bytes_per_step": int((o_E.numel() + o_U.numel() + o_X.numel() + o_V.numel() + o_dp.numel()
                                          + o_df.numel()) * 8 + o_cv.numel() * 4)}
        if abs(float(o_E[0]) - float(E[0])) > 1e-6:
            raise RuntimeError("host-buffer step disagrees with the device step: %r vs %r" % (float(o_E[0]), float(E[0])))
    elif not args.no_e2e:
        out_E = torch.empty(1, dtype=torch.float64).pin_memory()
        out_V = torch.empty(ctx.vavg_elems, dtype=torch.float64).pin_memory()
        out_df = torch.empty(3 * norb, dtype=torch.float64).pin_memory()
        out_dp = torch.empty(ctx.orb_elems, dtype=torch.float64).pin_memory()
        ke = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            pd = psi_h.to(dev, non_blocking=True)
            fd = fods_h.to(dev, non_blocking=True)
            E, Vavg, dpsi, dfod, _ = step(pd, fd)
            out_E.copy_(E, non_blocking=True)
            out_V.copy_(Vavg, non_blocking=True)
            out_df.copy_(dfod, non_blocking=True)
            out_dp.copy_(dpsi, non_blocking=True)
            torch.cuda.synchronize()
        barrier()
        te = D.max_over_ranks((time.perf_counter() - t0) / ke, dev)
        e2e = {"value": units / te, "unit": "solves/s",
               "h2d_bytes_per_step": int(psi_h.numel() * 8 + fods_h.numel() * 8),
               "d2h_bytes_per_step": int((out_E.numel() + out_V.numel() + out_df.numel() + out_dp.numel()) * 8)}

    # the plain float64 path on the same system (the comparison the metric
    # names), and the mixed path's deviation from it
    fp64 = None
    if prec == 1 and not args.no_fp64 and world == 1:
        E_m, Va_m, U_m, X_m = ctx.sic_energy_potential(psi, *step_outputs(ctx, psi, fods)[:2], 1.0)
        ctx64 = Context([s], precision=0, cg_tol=CG_TOL, preconditioner=pc)
        step64 = lambda: step_with(ctx64, psi, fods, gE)
        step64()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k64 = 2
        e0.record(stream)
        for _ in range(k64):
            o64 = step64()
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1) / k64
        phi64, V64 = step_outputs(ctx64, psi, fods)
        E_d, Va_d, U_d, X_d = ctx64.sic_energy_potential(psi, phi64, V64, 1.0)
        _, df_m = ctx.sic_backward(psi, fods, *step_outputs(ctx, psi, fods), gE, want_dpsi=False)
        _, df_d = ctx64.sic_backward(psi, fods, phi64, V64, gE, want_dpsi=False)
        rho_s = (psi.reshape(sum(s.norb), -1) ** 2)
        mask = torch.cat([rho_s[:s.norb[0]].sum(0), rho_s[s.norb[0]:].sum(0)]) > 1e-12
        fp64 = {"value": world * norb / (ms64 / 1e3), "unit": "solves/s", "ms_per_step": ms64, "steps": k64,
                "speedup_mixed_over_fp64": (world * norb / (ms_step / 1e3)) / (world * norb / (ms64 / 1e3)),
                "mixed_minus_fp64": {
                    "max_orbital_energy_Ha": float((U_m + X_m - U_d - X_d).abs().max().item()),
                    "E_sic_Ha": float((E_m - E_d).abs().max().item()),
                    "V_avg_maxabs_Ha": float((Va_m - Va_d).abs()[mask].max().item()),
                    "fod_gradient_max_Ha_per_bohr": float((df_m - df_d).abs().max().item())}}
        del ctx64

    # the same step with the multigrid-preconditioned CG inner solver, and
    # the roofline of its dominant kernel (the HBM-bound stencil apply)
    pcg = None
    if solver != 0 and prec == 1 and not args.no_pcg and world == 1:
        ctxp = Context([s], precision=1, cg_tol=CG_TOL, preconditioner=1, solver=0)
        for _ in range(2):
            step_with(ctxp, psi, fods, gE)
        barrier()
        ctxp.profile(True)
        ctxp.profile_read(reset=True)
        kp = 3
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kp):
            step_with(ctxp, psi, fods, gE)
        e1.record(stream)
        barrier()
        ms_p = D.max_over_ranks(e0.elapsed_time(e1), dev) / kp
        pp = ctxp.profile_read(reset=True)
        ctxp.profile(False)
        lp = max(pp["kernel_launches"], 1)
        ach_p = pp["kernel_bytes"] / (pp["kernel_ms"] / 1e3) / 1e9 if pp["kernel_ms"] > 0 else 0.0
        pcg = {"value": world * norb / (ms_p / 1e3), "unit": "solves/s", "ms_per_step": ms_p, "steps": kp,
               "roofline": {"bound": "hbm", "kernel": "k_apply12_tma<float>", "achieved": round(ach_p, 1),
                            "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": round(ach_p / peak, 4),
                            "traffic": (traffic_for(os.path.join(ROOT, "paper_2108_01186_gb300", "csrc",
                                                                 "stencil.cu"))
                                        if args.workload == "128" else None),
                            "alg_bytes_per_launch": pp["kernel_bytes"] / lp,
                            "avg_launch_ms": pp["kernel_ms"] / lp, "launches": pp["kernel_launches"],
                            "share_of_step": round(pp["kernel_ms"] / (ms_p * kp), 4)}}
        del ctxp

    # the two other real-size workloads, a few timed steps each (after the
    # 128^3 contexts are released)
    extra = {}
    if world == 1 and args.workload == "128" and not args.no_extra_workloads and prec == 1:
        del ctx
        torch.cuda.empty_cache()
        extra["uneven_batch"] = time_uneven(dev, stream, solver, steps=3)
        torch.cuda.empty_cache()
        extra["cube192"] = time_192(dev, stream, solver, steps=2)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "128":
        cpu = oracle_sample(s)

    if rank == 0:
        line = {"metric": METRIC if args.workload == "128" else METRIC_192, "value": value, "unit": "solves/s",
                "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak",
                "vs_baseline": None, "dtype": "f32-cg+f64" if prec == 1 else "f64", "data": "synthetic",
                "config": {"workload": workload, "precision": args.precision, "preconditioner": args.preconditioner,
                           "solver": args.solver,
                           "parallelism": ("orbitals of one system over %d ranks" % world if sharded
                                           else "one system per rank"),
                           "transforms": transforms_desc,
                           "cg_tol": CG_TOL,
                           "l2": "inputs larger than L2 (psi %.2f GB per rank)" % (8e-9 * norb * s.G),
                           "cg_iters_per_orbital_mean": float(np.mean(iters_sum) / args.steps)},
                "roofline": roof, "roofline_overlap": roof_ov, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e, "fp64_path": fp64,
                "pcg_path": pcg, **extra,
                "gpu_launches": prof["launches"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _timed(fn, steps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def time_uneven(dev, stream, solver, steps=3):
    """Forward step of the 64-system uneven batch (48^3..128^3, 2..40
    orbitals) in one context: solves/s."""
    import torch
    from paper_2108_01186_gb300 import synth
    from paper_2108_01186_gb300.flosic import Context
    systems = synth.make_uneven_batch(nsys=64, seed_base=2000)
    norb = sum(sum(x.norb) for x in systems)
    # blocks on the tensor-core transforms: sides multiples of 8 (<= 128) and a
    # 16-byte-aligned offset in the packed orbital arrays
    n_tc, off = 0, 0
    for x in systems:
        if x.n % 8 == 0 and x.n <= 128 and off % 4 == 0:
            n_tc += 1
        off += x.norb[0] * x.G
    ctx = Context(systems, precision=1, cg_tol=CG_TOL, preconditioner=1, solver=solver)
    psi = torch.tensor(np.concatenate([p.ravel() for x in systems for p in x.psi]), device=dev)
    fods = torch.tensor(np.concatenate([f.ravel() for x in systems for f in x.fods]), device=dev)
    del systems

    def fwd():
        phi, _, _ = ctx.build_flos(psi, fods, want_matrices=False)
        V, _, _ = ctx.orbital_poisson(phi)
        ctx.sic_energy_potential(psi, phi, V, 1.0)

    ms = _timed(fwd, steps, stream)
    out = {"metric": "orbital SIC solves/s, uneven batch, forward", "value": norb / (ms / 1e3),
           "unit": "solves/s", "ms_per_step": ms, "steps": steps,
           "workload": "64 systems, 48^3..128^3, h 0.15..0.3, 2..40 orbitals (%d orbitals in %d blocks; %d blocks "
                       "on the tensor-core transforms, the rest on the CUDA-core ones)"
                       % (norb, ctx.nblk, n_tc)}
    del ctx, psi, fods
    return out


def time_192(dev, stream, solver, steps=2):
    """Forward + adjoint step of 192^3, h = 0.15, 120 + 120 orbitals: solves/s."""
    import torch
    from paper_2108_01186_gb300 import synth
    from paper_2108_01186_gb300.flosic import Context
    s = synth.make_system(192, 0.15, 60, [120, 120], seed=4000)
    norb = sum(s.norb)
    ctx = Context([s], precision=1, cg_tol=CG_TOL, preconditioner=1, solver=solver)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), device=dev)
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods]), device=dev)
    del s
    gE = torch.ones(1, dtype=torch.float64, device=dev)
    ms = _timed(lambda: step_with(ctx, psi, fods, gE), steps, stream)
    out = {"metric": "orbital SIC solves/s at 192^3, forward + adjoint", "value": norb / (ms / 1e3),
           "unit": "solves/s", "ms_per_step": ms, "steps": steps,
           "workload": WORKLOAD_192,
           "device_gb_in_use": round((torch.cuda.mem_get_info(dev)[1] - torch.cuda.mem_get_info(dev)[0]) / 1e9, 1)}
    del ctx, psi, fods
    return out


def run_uneven(args):
    """Forward step of an uneven batch: 64 independent one-spin systems with
    grids 48^3..128^3 (h 0.15..0.3 bohr) and 2..40 orbitals, all in one
    context (every kernel launch covers every system)."""
    import torch
    from paper_2108_01186_gb300 import build, synth
    from paper_2108_01186_gb300 import dist as D
    from paper_2108_01186_gb300.flosic import Context
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D.init("nccl")
    build.build()
    systems = synth.make_uneven_batch(nsys=64, seed_base=2000 + 100000 * rank)
    norb = sum(sum(x.norb) for x in systems)
    solver = {"pcg": 0, "aar": 1, "kron": 2}[args.solver]
    ctx = Context(systems, precision=1, cg_tol=1e-10, preconditioner=1, solver=solver)
    dev = torch.device("cuda", local)
    psi = torch.tensor(np.concatenate([p.ravel() for x in systems for p in x.psi]), device=dev)
    fods = torch.tensor(np.concatenate([f.ravel() for x in systems for f in x.fods]), device=dev)
    del systems
    stream = torch.cuda.current_stream()

    def step():
        phi, _, _ = ctx.build_flos(psi, fods, want_matrices=False)
        V, iters, _ = ctx.orbital_poisson(phi)
        return ctx.sic_energy_potential(psi, phi, V, 1.0), iters

    for _ in range(args.warmup):
        step()
    D.barrier(torch.cuda.synchronize)
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, iters = step()
    e1.record(stream)
    D.barrier(torch.cuda.synchronize)
    clocks = clk.stop()
    ms = D.max_over_ranks(e0.elapsed_time(e1), dev) / args.steps
    if rank == 0:
        print(json.dumps({"metric": "orbital SIC solves/s, uneven batch (forward)", "value": world * norb / (ms / 1e3),
                          "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f32-cg+f64", "data": "synthetic",
                          "config": {"workload": "64 systems, 48^3..128^3, 2..40 orbitals (%d orbitals, %d spin blocks)"
                                     % (norb, ctx.nblk), "solver": args.solver,
                                     "cg_iters_per_orbital_mean": float(iters.float().mean().item())},
                          "clocks": clocks}), flush=True)
    D.barrier()


def run_fodopt(args):
    """FOD relaxation at 128^3 (32+32 orbitals): FIRE steps, each a forward
    step with warm-started Poisson solves plus the reverse mode for the FOD
    forces.  W untimed steps, then K timed steps."""
    import torch
    from paper_2108_01186_gb300 import build, fodopt, synth
    from paper_2108_01186_gb300 import dist as D
    from paper_2108_01186_gb300.flosic import Context
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D.init("nccl")
    build.build()
    s = synth.make_system(128, 0.2, 16, [32, 32], seed=3000 + rank)
    norb = sum(s.norb)
    solver = {"pcg": 0, "aar": 1, "kron": 2}[args.solver]
    ctx = Context([s], precision=1, cg_tol=1e-10, preconditioner=1, solver=solver)
    dev = torch.device("cuda", local)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), device=dev)
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods]), device=dev)
    stream = torch.cuda.current_stream()
    ev = {}
    fmax_hist = []

    def cb(k, x, E, fm, active):
        fmax_hist.append(float(fm[0]))
        if k == args.warmup or k == args.warmup + args.steps:
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            ev[k] = e

    D.barrier(torch.cuda.synchronize)
    clk = ClockSampler(local)
    clk.start()
    res = fodopt.optimize_fods(ctx, psi, fods, fmax=0.0, max_steps=args.warmup + args.steps, callback=cb)
    D.barrier(torch.cuda.synchronize)
    clocks = clk.stop()
    ms = D.max_over_ranks(ev[args.warmup].elapsed_time(ev[args.warmup + args.steps]), dev) / args.steps
    it = res["cg_iters"]
    if rank == 0:
        print(json.dumps({"metric": "FOD relaxation steps/s at 128^3 (forward + forces, warm-started Poisson)",
                          "value": world * 1e3 / ms, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32-cg+f64", "data": "synthetic",
                          "config": {"workload": "128^3 h=0.2, 32+32 orbitals, FIRE over 64 FODs",
                                     "solver": args.solver,
                                     "orbital_solves_per_s": world * norb * 1e3 / ms,
                                     "cg_iters_cold_first_step": it[0],
                                     "cg_iters_warm_mean": float(np.mean(it[args.warmup + 1:])),
                                     "max_force_first_last": [fmax_hist[0], fmax_hist[-1]]},
                          "clocks": clocks}), flush=True)
    D.barrier()


def measured_peaks():
    """MEASURED_PEAKS.json (driver-written), or the recipe's fallback figures."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def run_hamiltonian(args):
    """SC_AvgSIC Hamiltonian apply H psi = -1/2 Delta_h psi + V_avg psi on the
    128^3 workload's 32+32 orbitals (inputs in HBM, larger than L2)."""
    import torch
    from paper_2108_01186_gb300 import build, synth
    from paper_2108_01186_gb300 import dist as D
    from paper_2108_01186_gb300.flosic import Context
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D.init("nccl")
    build.build()
    s = synth.make_system(128, 0.2, 16, [32, 32], seed=3000 + rank)
    prec = 0 if args.precision == "fp64" else 1
    ctx = Context([s], precision=prec, cg_tol=1e-10, preconditioner=1)
    dev = torch.device("cuda", local)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), device=dev)
    vavg = torch.randn(ctx.vavg_elems, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(1)) * 0.1
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.hamiltonian_apply(psi, None, vavg, out)
    D.barrier(torch.cuda.synchronize)
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.hamiltonian_apply(psi, None, vavg, out)
    e1.record(stream)
    D.barrier(torch.cuda.synchronize)
    clocks = clk.stop()
    ms = D.max_over_ranks(e0.elapsed_time(e1), dev) / args.steps
    norb = sum(s.norb)
    alg = norb * s.G * 16 + ctx.nblk * s.G * 8          # psi in, H psi out, V_avg per spin block
    peaks = measured_peaks()
    ach = alg / (ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({"metric": "SC_AvgSIC Hamiltonian applies (orbitals/s) at 128^3", "value": world * norb * 1e3 / ms,
                          "unit": "orbitals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f32-ff" if prec else "f64", "data": "synthetic",
                          "config": {"workload": "128^3 h=0.2, 32+32 orbitals, H = -1/2 Lap + V_avg",
                                     "precision": args.precision},
                          "roofline": {"bound": "hbm", "kernel": "k_hamiltonian_ff" if prec else "k_hamiltonian64",
                                       "achieved": round(ach, 1), "peak": peaks.get("hbm_gbs"),
                                       "peak_source": peaks["source"],
                                       "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                                       "alg_bytes_per_launch": alg},
                          "clocks": clocks}), flush=True)
    D.barrier()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "fodopt":
        run_fodopt(args)
    elif args.workload == "hamiltonian":
        run_hamiltonian(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
