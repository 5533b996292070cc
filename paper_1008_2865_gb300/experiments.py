"""Sweeps of the model run as GPU batches, with the paper's observables.

  python -m paper_1008_2865_gb300.experiments sweep1024 [--steps 20000]
  python -m paper_1008_2865_gb300.experiments scan [--steps 500000] [--n 512]
  python -m paper_1008_2865_gb300.experiments interface [--steps 20000]

sweep1024: four 1024^2 periodic lattices, G1 = -5, G2 in {0, 0.3, 0.6, 0.9},
  rho = 0.7 (1 +- 1%) (seeds 2..5), FP32, one batched launch per step;
  aggregate MLUPS and GB/s, then droplet count, surface/volume, radius and the
  pseudo-energy ratios of each lattice.
scan: the A2 scan of Sec. 4 at fixed A1 = G1 + G2 = -4.9, A2 = G1 + (3/2) G2
  in {-4.9, -2.85, -0.8, 0.15, 0.65, 1.15, 1.65, 2.15, 2.65} (the values of
  Figs. 1, 3, 4), 512^2 lattices started from rho0 ln 2 (1 +- 1%), tau = 1;
  observables at log-spaced times (1e3 .. 5e5): droplet count, surface/volume,
  the radius R(t) of Eq. rad and E_surf / |E_bulk|; the growth exponent of
  R(t) ~ t^alpha fitted from t = 1e4 on (Fig. radius); the E/E_th, E_m/E_s and
  surface-share series of Figs. 5 and 7 from the trace.
interface: a flat liquid slab for each coupling pair of the scan (and the
  standard SC case), relaxed on a periodic 256 x 8 lattice: coexistence
  densities, the surface tension of Eq. gamma per interface and E_surf.

Each prints one JSON document. Synthetic seeded inputs only; the paper's own
figures are not reproduced, their quoted numbers are context.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import Batch, couplings_from_A, diag, inputs

A2_VALUES = (-4.9, -2.85, -0.8, 0.15, 0.65, 1.15, 1.65, 2.15, 2.65)
PAPER_RADII = {0.15: 30.0, 0.65: 8.0, 1.15: 6.5, 1.65: 5.1, 2.15: 4.4, 2.65: 3.9}


def _observe(b, i, shape):
    rho, _, _ = b.fields(i)
    try:
        e = b.energy(i)
    except Exception as exc:          # a lattice that went non-finite
        return {"error": str(exc)}
    return diag.summary(rho, e)


def sweep1024(steps=20000, n=1024, g2s=(0.0, 0.3, 0.6, 0.9), trace_every=100):
    import torch

    rhos = [inputs.noisy_density(n, n, 2 + i, mean=0.7, amp=0.01, mode="rel")
            for i in range(len(g2s))]
    stream = torch.cuda.current_stream()
    out = {"workload": f"{len(g2s)} x {n}^2, G1=-5, G2 in {list(g2s)}, rho=0.7(1+-1%), "
                       f"{steps} steps, FP32, batched", "lattices": []}
    with Batch(rhos, G1=-5.0, G2=list(g2s), trace_every=trace_every,
               stream=stream.cuda_stream) as b:
        b.step(trace_every)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps - trace_every)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sites = len(g2s) * n * n
        out["mlups"] = sites * (steps - trace_every) / (ms / 1e3) / 1e6
        out["gb_per_s"] = out["mlups"] * 1e6 * 80 / 1e9
        for i, g2 in enumerate(g2s):
            rec = {"G2": g2}
            rec.update(_observe(b, i, (n, n)))
            tr = b.trace(i)
            rec["mass_drift"] = float(abs(tr[-1, 1] - tr[0, 1]) / tr[0, 1])
            out["lattices"].append(rec)
    return out


SNAPSHOTS = (1000, 2000, 5000, 10000, 20000, 50000, 100000, 200000, 500000)


def _decimate(series, points=60):
    """At most `points` rows of each array in a dict, evenly spaced, last row kept."""
    n = len(series["t"])
    if n <= points:
        idx = np.arange(n)
    else:
        idx = np.unique(np.append(np.linspace(0, n - 1, points).astype(int), n - 1))
    return {k: [float(v) for v in np.asarray(a)[idx]] for k, a in series.items()}


def scan(steps=500000, n=512, a2_values=A2_VALUES, A1=-4.9, snapshots=SNAPSHOTS,
         trace_every=1000, fit_from=10000):
    import torch

    pairs = [couplings_from_A(A1, a2) for a2 in a2_values]
    rho_c = math.log(2.0)
    rhos = [inputs.noisy_density(n, n, 500 + i, mean=rho_c, amp=0.01, mode="rel")
            for i in range(len(a2_values))]
    stream = torch.cuda.current_stream()
    out = {"workload": f"A1={A1}, A2 scan {list(a2_values)} (G2 = 2 (A2 - A1), G1 = A1 - G2), "
                       f"{n}^2, rho = ln2 (1 +- 1%), tau = 1, FP32, batched",
           "couplings": [{"A2": a2, "G1": g1, "G2": g2} for a2, (g1, g2) in zip(a2_values, pairs)],
           "snapshots": {}}
    t0 = time.perf_counter()
    with Batch(rhos, G1=[p[0] for p in pairs], G2=[p[1] for p in pairs],
               trace_every=trace_every, stream=stream.cuda_stream) as b:
        marks = sorted({s for s in snapshots if s < steps} | {steps})
        done = 0
        for m in marks:
            b.step(m - done)
            done = m
            torch.cuda.synchronize()
            rows = []
            for i, a2 in enumerate(a2_values):
                rec = {"A2": a2}
                rec.update(_observe(b, i, (n, n)))
                rho, _, _ = b.fields(i)
                g1, g2 = pairs[i]
                if "error" not in rec:
                    eb = b.energy(i)[2]
                    rec["E_surf_over_abs_E_bulk"] = diag.surface_energy(rho, g1, g2) / abs(eb)
                if m == steps and a2 in PAPER_RADII:
                    rec["paper_radius"] = PAPER_RADII[a2]
                rows.append(rec)
            out["snapshots"][str(m)] = rows
        # R(t), droplet count and surface/volume per A2 across the snapshots, and
        # the growth exponent of R(t) ~ t^alpha from fit_from on (Fig. radius)
        out["series"] = []
        for i, a2 in enumerate(a2_values):
            ts = [int(m) for m in marks]
            R = [out["snapshots"][str(m)][i].get("radius", float("nan")) for m in marks]
            rec = {"A2": a2, "t": ts, "R": R,
                   "droplets": [out["snapshots"][str(m)][i].get("droplets") for m in marks],
                   "surface_to_volume": [out["snapshots"][str(m)][i].get("surface_to_volume")
                                         for m in marks]}
            late = [(t, r) for t, r in zip(ts, R) if t >= fit_from]
            rec["alpha_from_%d" % fit_from] = (diag.growth_exponent(*zip(*late))
                                               if len(late) >= 2 else None)
            tr = b.trace(i)
            rec["energy_series"] = _decimate(diag.energy_series(tr, n * n)) if len(tr) else None
            out["series"].append(rec)
        out["traces_Em_over_Es_last"] = []
        for i in range(len(a2_values)):
            tr = b.trace(i)
            out["traces_Em_over_Es_last"].append(float(tr[-1, 3] / tr[-1, 2]) if len(tr) else None)
    torch.cuda.synchronize()
    out["wall_s"] = time.perf_counter() - t0
    out["site_updates"] = len(a2_values) * n * n * steps
    out["mlups"] = out["site_updates"] / out["wall_s"] / 1e6
    return out


def interface(steps=20000, nx=256, ny=8, A1=-4.9, a2_values=A2_VALUES, extra=((-5.0, 0.0),)):
    """Flat interfaces: a liquid slab (columns nx/4 .. 3nx/4) relaxed for `steps` steps
    for each (G1, G2) of the A2 scan plus `extra` pairs, FP32, one batch. Per lattice:
    the coexistence densities (the slab's centre and the gas far from it), the
    surface tension of Eq. gamma per interface from the y-averaged psi profile,
    and E_surf = -(A1/12) sum |grad psi|^2 against E - E_bulk of the lattice sums."""
    import torch

    pairs = [couplings_from_A(A1, a2) for a2 in a2_values] + [tuple(p) for p in extra]
    x = np.arange(nx) + 0.5
    prof = 0.2 + 1.6 * 0.5 * (np.tanh((x - nx / 4) / 3) - np.tanh((x - 3 * nx / 4) / 3))
    rho0 = np.ascontiguousarray(prof[None, :].repeat(ny, 0))
    stream = torch.cuda.current_stream()
    out = {"workload": f"flat slab on {nx} x {ny} periodic lattices, {steps} steps, FP32, "
                       f"tau = 1; couplings of the A1 = {A1} scan and {list(extra)}",
           "interfaces": []}
    with Batch([rho0] * len(pairs), G1=[p[0] for p in pairs], G2=[p[1] for p in pairs],
               trace_every=0, stream=stream.cuda_stream) as b:
        b.step(steps)
        torch.cuda.synchronize()
        for i, (g1, g2) in enumerate(pairs):
            rho, _, _ = b.fields(i)
            try:
                es, em, eb, _ = b.energy(i)
            except Exception as exc:
                out["interfaces"].append({"G1": g1, "G2": g2, "error": str(exc)})
                continue
            col = rho.mean(axis=0)
            psi = diag.psi_of(col)
            out["interfaces"].append({
                "G1": g1, "G2": g2, "A2": g1 + 1.5 * g2, "G1+12/7G2": g1 + 12.0 / 7.0 * g2,
                "rho_liquid": float(col[nx // 2]), "rho_gas": float(col[0]),
                "flat": bool(np.max(np.abs(rho - col[None, :])) < 1e-3 * float(col.max())),
                "gamma": diag.surface_tension(psi, g1, g2),
                "E_surf": diag.surface_energy(rho, g1, g2),
                "E_minus_E_bulk": es + em - eb})
    return out


def _json_default(o):
    if isinstance(o, (np.floating, np.integer)):
        return o.item()
    raise TypeError(type(o))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["sweep1024", "scan", "interface"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--n", type=int, default=None)
    args = ap.parse_args()
    if args.which == "sweep1024":
        res = sweep1024(steps=args.steps or 20000, n=args.n or 1024)
    elif args.which == "interface":
        res = interface(steps=args.steps or 20000)
    else:
        res = scan(steps=args.steps or 500000, n=args.n or 512)
    print(json.dumps(res, default=_json_default, indent=1))


if __name__ == "__main__":
    main()
