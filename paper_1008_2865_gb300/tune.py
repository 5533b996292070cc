"""Launch-shape autotuner for the fused step kernel.

The fused kernel's only free parameters are the CTA width (block_x threads =
block_x - 2 output columns plus a one-column halo on each side) and the
number of output rows a CTA marches over. Narrow CTAs waste a larger share of
lanes on halo columns; short row chunks re-read more halo rows; tall chunks
give too few CTAs for the 152 SMs. The tuner times every candidate on the
real lattice shape with CUDA events and keeps the fastest in a JSON cache
keyed by GPU name, lattice shape and storage precision.

  python -m paper_1008_2865_gb300.tune 8192 8192 [fp32]
"""
from __future__ import annotations

import json
import os
import sys
import threading

BLOCK_X = (64, 96, 128, 192, 256)
BULK_BLOCK_X = (64, 128, 256)
ROWS = (4, 8, 16, 24, 32, 48, 56, 64, 72, 80, 96, 128, 192, 256, 384)
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_launch.json")
_lock = threading.Lock()


def _gpu_name(device=0):
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return "unknown"


def _key(nx, ny, prec, device=0):
    return f"{_gpu_name(device)}|{nx}x{ny}|{prec}"


def _load_cache():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def lookup(nx, ny, prec="fp32", device=0):
    """Cached (block_x, rows_per_cta, pipeline) for this GPU and shape, or None."""
    rec = _load_cache().get(_key(nx, ny, prec, device))
    return tuple(rec["best"]) if rec else None


def candidates(nx, ny):
    """(block_x, rows_per_cta, pipeline) shapes; the library rejects the ones a
    lattice cannot use (the bulk-copy pipeline needs aligned, wide rows)."""
    out = []
    for pipe, bxs in ((0, BLOCK_X), (1, BULK_BLOCK_X)):
        for bx in bxs:
            for rows in ROWS:
                if rows > max(16, ny):
                    continue
                out.append((bx, rows, pipe))
    return out


def tune(nx, ny, prec="fp32", steps=20, device=0, save=True, G1=-5.0, G2=0.6):
    """Time each candidate shape for `steps` steps (including the reduction steps of a
    10-step trace period) and return ((block_x, rows), {shape: ms_per_step})."""
    import torch

    from . import Lattice, inputs

    rho0 = inputs.noisy_density(nx, ny, seed=7, mean=0.7, amp=0.01, mode="rel")
    stream = torch.cuda.current_stream(device)
    table = {}
    with Lattice(rho0, G1=G1, G2=G2, prec=prec, trace_every=10, device=device,
                 stream=stream.cuda_stream) as lat:
        for bx, rows, pipe in candidates(nx, ny):
            try:
                lat.set_launch(bx, rows, pipe)
            except Exception:
                continue
            lat.step(3)
            lat.step((-lat.t) % 10)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            e1.synchronize()
            table[(bx, rows, pipe)] = e0.elapsed_time(e1) / steps
    best = min(table, key=table.get)
    if save:
        with _lock:
            cache = _load_cache()
            cache[_key(nx, ny, prec, device)] = {
                "best": list(best), "ms_per_step": table[best],
                "mlups": nx * ny / (table[best] / 1e3) / 1e6,
                "candidates": {f"{b},{r},{p}": round(v, 5) for (b, r, p), v in sorted(table.items())},
            }
            tmp = CACHE + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(cache, fh, indent=1, sort_keys=True)
            os.replace(tmp, CACHE)
    return best, table


def _batch_key(shapes, prec, device=0):
    import hashlib
    h = hashlib.sha1(repr(sorted(shapes)).encode()).hexdigest()[:12]
    return f"{_gpu_name(device)}|batch:{len(shapes)}:{h}|{prec}"


def lookup_batch(shapes, prec="fp32", device=0):
    """Cached (block_x, rows_per_cta) for a batch of these lattice shapes, or None."""
    rec = _load_cache().get(_batch_key(shapes, prec, device))
    return tuple(rec["best"]) if rec else None


def tune_batch(rho_list, G2_list, prec="fp32", steps=20, device=0, save=True, G1=-5.0):
    """Time each tile shape for a batch (one launch per step over all replicas, graph
    replay) and return ((block_x, rows), {shape: ms_per_step})."""
    import torch

    from . import Batch

    stream = torch.cuda.current_stream(device)
    shapes = [tuple(r.shape) for r in rho_list]
    sites = sum(a * b for a, b in shapes)
    table = {}
    with Batch(rho_list, G1=G1, G2=list(G2_list), prec=prec, trace_every=10, device=device,
               stream=stream.cuda_stream) as b:
        for bx in BLOCK_X:
            for rows in (8, 12, 16, 24, 32, 48, 64):
                try:
                    b.set_launch(bx, rows, 1)
                except Exception:
                    continue
                b.step(10)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.step(steps)
                e1.record(stream)
                e1.synchronize()
                table[(bx, rows)] = e0.elapsed_time(e1) / steps
    best = min(table, key=table.get)
    if save:
        with _lock:
            cache = _load_cache()
            cache[_batch_key(shapes, prec, device)] = {
                "best": list(best), "ms_per_step": table[best],
                "mlups": sites / (table[best] / 1e3) / 1e6,
                "candidates": {f"{b},{r}": round(v, 5) for (b, r), v in sorted(table.items())},
            }
            tmp = CACHE + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(cache, fh, indent=1, sort_keys=True)
            os.replace(tmp, CACHE)
    return best, table


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "batch":
    # the 96-replica G2 sweep: 32 each of 192^2, 384^2, 640^2
    from . import inputs
    sizes = [n for n in (192, 384, 640) for _ in range(32)]
    g2 = inputs.g2_sweep(len(sizes), seed=100)
    rhos = [inputs.noisy_density(n, n, 1000 + i, mean=0.7, amp=0.01, mode="rel")
            for i, n in enumerate(sizes)]
    best, table = tune_batch(rhos, g2)
    for k in sorted(table, key=table.get)[:8]:
        print(k, f"{table[k]:.4f} ms/step")
    print("best", best)
elif __name__ == "__main__":
    nx = int(sys.argv[1]) if len(sys.argv) > 1 else 8192
    ny = int(sys.argv[2]) if len(sys.argv) > 2 else nx
    prec = sys.argv[3] if len(sys.argv) > 3 else "fp32"
    best, table = tune(nx, ny, prec)
    for k in sorted(table, key=table.get)[:8]:
        print(k, f"{table[k]:.4f} ms/step", f"{nx * ny / table[k] / 1e3:.0f} MLUPS")
    print("best", best)
