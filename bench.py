"""Benchmark: MLUPS of the fused FP32 two-belt Shan–Chen step on GB300.

One "step" is one pass of the whole hot path over the lattice: moments,
psi, the two-belt force, velocity-shifted BGK collision, streaming (on chip),
psi of the next state, and (every 10th step) the fused pseudo-energy and mass
reduction. The workload is the 8192 x 8192 periodic lattice, FP32, G1 = -5,
G2 = 0.6, rho = 0.7 (1 +- 1%) seeded noise — the bandwidth-roofline case.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line. With --impl reference, the FP64 CPU oracle is timed on
the host cores on a bounded sample of the same workload (each step one full
step of a 512 x 512 periodic lattice with the same parameters and noise).
Under torchrun (N > 1) each rank runs its own replica of the lattice on its
own GPU (independent replicas, no data exchange); value = all ranks' site
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 8192
G1, G2, OMEGA, SEED = -5.0, 0.6, 1.0, 7
TRACE_EVERY = 10
BYTES_PER_SITE = 80          # 36 B populations in + 36 B out + 4 B dpsi in + 4 B dpsi out
METRIC = "MLUPS and % HBM roofline (FP32 fused step, 1 GB300); adjoint+batched vs plain"
WORKLOAD = ("{n}x{n} periodic D2Q9 two-belt Shan-Chen, FP32 (deviation storage), omega=1, "
            "G1=-5.0, G2=0.6, rho=0.7(1+-1%) seeded uniform noise (seed 7), energy+mass "
            "reduction every 10 steps")


def _dist():
    from paper_1008_2865_gb300 import replicas
    return replicas.world()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy test)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, earlier GB300 copy measurement)"


def _sources_sha256():
    """Hashes of the sources the timed step kernel (k_step) is built from."""
    out = {}
    for name in ("lb_fp32.cu", "lb_device.cuh", "lb_internal.h"):
        path = os.path.join(ROOT, "paper_1008_2865_gb300", "csrc", name)
        with open(path, "rb") as fh:
            out[name] = hashlib.sha256(fh.read()).hexdigest()
    return out


def _traffic_record(nx, ny, launch):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if the
    kernel sources and launch shape are unchanged since it was taken (else None)."""
    rec_path = os.path.join(ROOT, "profiles", "step_fp32_traffic.json")
    try:
        with open(rec_path) as fh:
            rec = json.load(fh)
        if (rec.get("sources_sha256") == _sources_sha256() and rec.get("nx") == nx
                and rec.get("ny") == ny and list(rec.get("launch", [])) == list(launch)):
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


BATCH_SIZES = (192, 384, 640)
BATCH_PER_SIZE = 32


def run_batched(steps, warmup, stream, dev):
    """The 96-replica G2 sweep (32 each of 192^2, 384^2, 640^2; G2 ~ U[0, 1) seed 100;
    seeds 1000..1095; G1 = -5, FP32): aggregate MLUPS of the batched launch (one launch
    per step over all replicas, CUDA-graph replay) against running the same replicas
    one after another, each a single-lattice state stepping on its own."""
    import torch

    from paper_1008_2865_gb300 import Batch, Lattice, inputs
    sizes = [n for n in BATCH_SIZES for _ in range(BATCH_PER_SIZE)]
    g2 = inputs.g2_sweep(len(sizes), seed=100)
    rhos = [inputs.noisy_density(n, n, 1000 + i, mean=0.7, amp=0.01, mode="rel")
            for i, n in enumerate(sizes)]
    sites = sum(n * n for n in sizes)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    from paper_1008_2865_gb300 import tune
    shape = tune.lookup_batch([r.shape for r in rhos]) or (128, 32)
    with Batch(rhos, G1=G1, G2=list(g2), trace_every=TRACE_EVERY, device=dev,
               stream=stream.cuda_stream) as b:
        b.set_launch(shape[0], shape[1], 1)
        b.step(max(warmup, 3) * TRACE_EVERY)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms_batch = e0.elapsed_time(e1)
        launch = b.launch
    lats = [Lattice(r, G1=G1, G2=float(g), trace_every=TRACE_EVERY, device=dev,
                    stream=stream.cuda_stream) for r, g in zip(rhos, g2)]
    for lat in lats:
        lat.step(max(warmup, 3) * TRACE_EVERY)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for lat in lats:
        lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for lat in lats:
        lat.close()
    return {"workload": "96 replicas: 32 each of 192^2, 384^2, 640^2 periodic lattices, "
                        "G2 ~ U[0,1) (seed 100), seeds 1000..1095, G1=-5, FP32, trace every 10",
            "sites": sites, "steps": steps,
            "mlups": sites * steps / (ms_batch / 1e3) / 1e6,
            "one_by_one_mlups": sites * steps / (ms_seq / 1e3) / 1e6,
            "speedup_vs_one_by_one": ms_seq / ms_batch,
            "launch": {"block_x": launch[0], "rows_per_cta": launch[1], "cuda_graph": bool(launch[2])},
            "launches_per_step": "1 (+1 per-replica reduction every 10 steps)"}


def run_adjoint(stream, dev, T=2000, n=512):
    """The adjoint workload: 512^2 periodic FP32, G1 = -5, G2 = 0.5, T = 2000 steps with
    ceil(sqrt(T)) checkpointing; J = pseudo-energy at T + misfit to a seeded target.
    Time of lb_adjoint (forward with checkpoints + recomputation + reverse sweep, its
    working memory included) against T plain steps of the same lattice."""
    import math

    import torch

    from paper_1008_2865_gb300 import Lattice, inputs
    r0 = inputs.noisy_density(n, n, 11, mean=0.7, amp=0.01, mode="rel")
    tgt = torch.from_numpy(inputs.noisy_density(n, n, 12, mean=0.7, amp=0.01, mode="rel")).cuda()
    grad = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {}
    for rep in range(2):            # the first pass warms up allocations and module loads
        with Lattice(r0, G1=G1, G2=0.5, trace_every=0, device=dev, stream=stream.cuda_stream) as lat:
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            lat.step(T)
            e1.record(stream)
            e1.synchronize()
            res["forward_ms"] = e0.elapsed_time(e1)
        with Lattice(r0, G1=G1, G2=0.5, trace_every=0, device=dev, stream=stream.cuda_stream) as lat:
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            J, _, gG = lat.adjoint(T, tgt, grad_rho=grad)
            e1.record(stream)
            e1.synchronize()
            res["adjoint_ms"] = e0.elapsed_time(e1)
    return {"workload": f"{n}x{n} periodic FP32 (FP64 gradient accumulation), G1=-5, G2=0.5, "
                        f"T={T}, checkpoint every {math.ceil(math.sqrt(T))} steps; "
                        "J = E_s(T) + E_m(T) + sum (rho(T) - rho*)^2, rho* seeded (seed 12)",
            "forward_ms": res["forward_ms"], "adjoint_ms": res["adjoint_ms"],
            "adjoint_over_forward": res["adjoint_ms"] / res["forward_ms"],
            "J": J, "dJ_dG1": gG[0], "dJ_dG2": gG[1],
            "includes": "forward with checkpoints, per-segment recomputation, reverse sweep "
                        "(2 kernels per step), gradient w.r.t. rho_init, G1, G2"}


def run_fp16(steps, warmup, stream, dev, peak):
    """The same 8192^2 workload with the populations stored as FP16 deviations (44 B per
    site: 18 B read + 18 B written + 4 + 4 B of psi), FP32 arithmetic: device-resident
    MLUPS and the fraction of the copy bandwidth at 44 B/site."""
    import torch

    from paper_1008_2865_gb300 import Lattice, inputs, tune
    rho0 = inputs.noisy_density(NX, NY, SEED, mean=0.7, amp=0.01, mode="rel")
    with Lattice(rho0, omega=OMEGA, G1=G1, G2=G2, prec="fp16_delta", trace_every=TRACE_EVERY,
                 device=dev, stream=stream.cuda_stream) as lat:
        best = tune.lookup(NX, NY, "fp16_delta")
        if best and len(best) == 3:
            lat.set_launch(*best)
        lat.step(warmup)
        lat.step((-lat.t) % TRACE_EVERY)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        launch = lat.launch
        e = lat.energy()
        if not all(np.isfinite(e)):
            raise RuntimeError(f"non-finite FP16-storage energies {e}")
    gbs = 44 * NX * NY / (ms / 1e3) / 1e9
    return {"workload": WORKLOAD.format(n=NX).replace("FP32 (deviation storage)",
                                                      "FP16 deviation storage, FP32 arithmetic"),
            "mlups": NX * NY / (ms / 1e3) / 1e6, "ms_per_step": ms, "steps": steps,
            "launch": {"block_x": launch[0], "rows_per_cta": launch[1],
                       "pipeline": ["register-prefetch", "bulk-copy rings"][launch[2]]},
            "roofline": {"bound": "hbm", "bytes_per_site": 44, "achieved": gbs, "peak": peak,
                         "unit": "GB/s", "frac": gbs / peak,
                         "roof_mlups": peak * 1e9 / 44 / 1e6}}


def run_step_split(stream, dev, launch, steps=20):
    """Time of a plain step and of a step with the fused energy/mass reduction, each
    timed over `steps` consecutive steps of the 8192^2 FP32 lattice (trace_every = 0
    and 1), with the benchmark's launch shape."""
    import torch

    from paper_1008_2865_gb300 import Lattice, inputs
    rho0 = inputs.noisy_density(NX, NY, SEED, mean=0.7, amp=0.01, mode="rel")
    out = {}
    for name, te in (("plain", 0), ("reduce", 1)):
        with Lattice(rho0, omega=OMEGA, G1=G1, G2=G2, trace_every=te, device=dev,
                     stream=stream.cuda_stream) as lat:
            lat.set_launch(*launch)
            lat.step(3)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            e1.synchronize()
            out[name + "_ms"] = e0.elapsed_time(e1) / steps
    out["reduce_over_plain"] = out["reduce_ms"] / out["plain_ms"]
    return out


def cpu_baseline(seconds=12.0):
    """Oracle MLUPS on the host cores: a 512x512 lattice of the workload's parameters."""
    import oracle
    from paper_1008_2865_gb300 import inputs
    n = 512
    rho0 = inputs.noisy_density(n, n, SEED, mean=0.7, amp=0.01, mode="rel")
    t0 = time.perf_counter()
    oracle.run(rho0, 4, omega=OMEGA, G1=G1, G2=G2)
    per_step = max((time.perf_counter() - t0) / 4, 1e-4)
    steps = max(4, min(2000, int(seconds / per_step)))
    t0 = time.perf_counter()
    oracle.run(rho0, steps, omega=OMEGA, G1=G1, G2=G2, trace_every=TRACE_EVERY)
    dt = time.perf_counter() - t0
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{n}x{n} periodic lattice, same parameters and noise, {steps} steps "
                      f"(FP64 oracle, OpenMP over rows), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1008_2865_gb300 import inputs
    n = 512
    rho0 = inputs.noisy_density(n, n, SEED, mean=0.7, amp=0.01, mode="rel")
    f = oracle.init(rho0)
    for _ in range(args.warmup):
        f = oracle.step(f, omega=OMEGA, G1=G1, G2=G2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(f, omega=OMEGA, G1=G1, G2=G2)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 noise)", "impl": "reference",
            "config": {"workload": WORKLOAD.format(n=NX), "sample": f"{n}x{n} periodic lattice per step"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": f"each step one full step of a {n}x{n} lattice"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    from paper_1008_2865_gb300 import Lattice, capi, inputs

    from paper_1008_2865_gb300 import replicas

    ws, rank, local = _dist()
    if ws > 1:
        replicas.init("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    capi.load(build_if_missing=True)
    stream = torch.cuda.current_stream()

    NX = NY = args.size
    rho0 = inputs.noisy_density(NX, NY, replicas.seed_for_rank(SEED, rank), mean=0.7, amp=0.01,
                                mode="rel")

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, device="cuda")

    # ---- device-resident timing: inputs already in HBM
    lat = Lattice(rho0, omega=OMEGA, G1=G1, G2=G2, prec=args.prec, trace_every=TRACE_EVERY,
                  device=dev, stream=stream.cuda_stream)
    if args.launch:
        lat.set_launch(*(int(v) for v in args.launch.split(",")))
    elif args.prec != "fp64":
        from paper_1008_2865_gb300 import tune
        best = tune.lookup(NX, NY, args.prec)
        if best and len(best) == 3:
            lat.set_launch(*best)
    lat.step(args.warmup)
    # align the timed region to a trace period so it holds K/10 reduction steps
    lat.step((-lat.t) % TRACE_EVERY)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        time.sleep(0.3)
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    launch = lat.launch
    e = lat.energy()
    if not all(np.isfinite(e)):
        raise RuntimeError(f"non-finite energies {e}")
    lat.close()
    del lat
    torch.cuda.synchronize()

    N = NX * NY
    value = N * args.steps * ws / (ms_max / 1e3) / 1e6
    per_launch_s = ms / 1e3 / args.steps
    peak, peak_src = _peaks()
    achieved = (BYTES_PER_SITE if args.prec == "fp32" else 44) * N / per_launch_s / 1e9
    traffic = _traffic_record(NX, NY, launch)
    bytes_per_site = BYTES_PER_SITE if args.prec == "fp32" else 44

    if args.skip_e2e:
        print(json.dumps({"size": NX, "prec": args.prec, "launch": launch, "MLUPS": value,
                          "ms_per_step": ms / args.steps,
                          "GBs": bytes_per_site * N / per_launch_s / 1e9}))
        return 0

    # ---- end to end through the public API with host buffers
    pinned_in = torch.from_numpy(rho0).pin_memory()
    pinned_out = torch.empty((NY, NX), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    lat2 = Lattice(pinned_in, omega=OMEGA, G1=G1, G2=G2, prec=args.prec,
                   trace_every=TRACE_EVERY, device=dev, stream=stream.cuda_stream)
    lat2.set_launch(*launch)
    lat2.step(args.steps)
    rows_read = len(lat2.trace())
    lat2.fields(rho=pinned_out)
    torch.cuda.synchronize()
    dt_e2e = max_over_ranks(time.perf_counter() - t0)
    lat2.close()
    e2e_value = N * args.steps * ws / dt_e2e / 1e6

    batched = run_batched(args.steps, args.warmup, stream, dev) if not args.skip_batch else None
    adjoint = run_adjoint(stream, dev) if not args.skip_batch else None
    fp16 = run_fp16(args.steps, args.warmup, stream, dev, peak) if not args.skip_batch else None
    split = run_step_split(stream, dev, launch) if not args.skip_batch else None

    out = None
    if rank == 0:
        cpu = cpu_baseline() if ws == 1 else None
        if batched is not None:
            batched["vs_plain_mlups"] = batched["mlups"] / value
        clocks = clk.summary()
        out = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32" else "f32 (f16 storage)",
            "data": "synthetic (seeded SplitMix64 noise)",
            "config": {"workload": WORKLOAD.format(n=NX), "nx": NX, "ny": NY,
                       "l2": "state 5.4 GB per replica >> 129 MB L2; no flush needed",
                       "launch": {"block_x": launch[0], "rows_per_cta": launch[1],
                                  "pipeline": ["register-prefetch", "bulk-copy rings"][launch[2]]},
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "kernel": ("k_step_bulk (one launch per step)" if launch[2] else
                                    "k_step (one launch per step; a reduction step adds "
                                    "k_step_total, its grid sum)"),
                         "bytes_per_site": bytes_per_site},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": 8 * N / args.steps,
                    "d2h_bytes_per_step": (8 * N + 40 * rows_read) / args.steps,
                    "includes": "lb_init from pinned host rho (H2D), lb_step(K), lb_trace of the "
                                "K/10 trace rows (t, mass, E_s, E_m, E_bulk) (D2H), lb_fields rho "
                                "to pinned host (D2H)"},
            # one step kernel per step; the register-prefetch pipeline's reduction steps
            # (t % TRACE_EVERY == 0; the timed region starts at such a t) add k_step_total
            "gpu_launches": args.steps + (0 if launch[2] else -(-args.steps // TRACE_EVERY)),
            "clocks": clocks,
            "batched": batched,
            "adjoint": adjoint,
            "fp16_delta": fp16,
            "step_split": split,
        }
    if ws > 1:
        import torch.distributed as dist
        replicas.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=8192,
                    help="lattice side (profiling of smaller cases; the benchmark is 8192)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp16_delta"])
    ap.add_argument("--launch", default=None, help="block_x,rows_per_cta,pipeline override")
    ap.add_argument("--skip-e2e", action="store_true",
                    help="time the device-resident steps only and print a short line")
    ap.add_argument("--skip-batch", action="store_true",
                    help="leave out the batched sweep, the adjoint, the FP16-storage run and "
                         "the plain/reduce split")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
