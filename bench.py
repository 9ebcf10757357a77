#!/usr/bin/env python3
"""Benchmark of the hot path: the nDGP (Vainshtein) multigrid field solve of
MG-GLAM (arXiv:2110.00566, Sec. 3.2) on a 512^3 periodic mesh.

Workload (synthetic, seeded): 256^3 particles in a 256 Mpc/h box, displaced
from a lattice by the Zel'dovich field of P(k) = A k^0.96 exp(-k/5) with
sigma_8 = 0.8 evaluated at z = 0 (seed 2 + rank), deposited by CIC on the
512^3 mesh; a = 1, Omega_m = 0.3, H0 r_c = 1.  One step = one complete
solve from phi = 0 to eps/eps_ref < 1e-8 with V(2,2) cycles (source prep,
all cycles, gauge fix), inputs resident in HBM.  The metric is smoother
cell-updates (summed over all levels and cycles) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Under torchrun each rank solves its own independent instance (replicas:
weak scaling, no data-path collective); value sums the ranks' cell-updates
over the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nDGP MG-solve Gcell-updates/s @512^3"
UNIT = "Gcell-updates/s"
HBM_PEAK_FALLBACK = 6800.0


def args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--ng", type=int, default=512)
    p.add_argument("--np", type=int, default=256)
    p.add_argument("--box", type=float, default=256.0)
    p.add_argument("--rc", type=float, default=1.0)
    p.add_argument("--rtol", type=float, default=1e-8)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def particles(a, rank):
    from paper_2110_00566_gb300 import inputs
    pk = inputs.pk_cutoff(0.96, 5.0, 0.8)
    pos, _ = inputs.zeldovich(a.np, a.ng, a.box, pk, 1.0, seed=2 + rank)
    return pos


class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(delta_host, a, sample_cycles=1):
    """The FP64 oracle as it stands, on the same delta: one V(2,2) cycle of
    the solve (initial residual, the cycle, final residual and gauge),
    OpenMP over all host cores."""
    import oracle
    s0, eps_ref, alpha, _ = oracle.dgp_source(delta_host, 1.0, 0.3, a.rc)
    op = oracle.dgp_op(alpha)
    t = time.perf_counter()
    u, st = oracle.mg_solve(op, s0, eps_ref, oracle.Opts(rtol=0.0, max_cycles=sample_cycles))
    dt = time.perf_counter() - t
    ng = a.ng
    per_cycle = 0
    n = ng
    levels = oracle.num_levels(ng)
    for l in range(levels):
        cells = (ng >> l) ** 3
        per_cycle += (64 if l == levels - 1 else 4) * cells
    updates = per_cycle * st.cycles
    return {"value": updates / dt / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d V(2,2) cycle(s) of the %d^3 solve (with its initial and final residual passes), "
                      "plain C FP64 oracle, OpenMP over i-planes" % (st.cycles, ng),
            "seconds": dt}


def run_reference(a, rank, world):
    if rank != 0:
        return
    import numpy as np
    import oracle
    pos = particles(a, 0)
    delta, _ = oracle.cic_deposit(pos, a.ng, a.np)
    vals = []
    for _ in range(a.warmup):
        pass                                    # the oracle has no warm-up state
    t0 = time.perf_counter()
    for _ in range(a.steps):
        cb = cpu_baseline(delta, a)
        vals.append(cb["value"])
    dt = time.perf_counter() - t0
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "nDGP FAS V(2,2) solve, %d^3 mesh, CIC of %d^3 Zel'dovich particles, L=%g Mpc/h, "
                                   "a=1, Omega_m=0.3, H0 rc=%g" % (a.ng, a.np, a.box, a.rc),
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        import __graft_entry__
        from oracle import build as ob
        ob.build()
        return run_reference(a, rank, world)

    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2110_00566_gb300 import binding as B

    ctx = B.Context(local, torch.cuda.current_stream(dev))
    ng = a.ng
    pos = torch.from_numpy(particles(a, rank)).to(dev)
    delta = torch.empty((ng, ng, ng), dtype=torch.float64, device=dev)
    B.pm_cic_deposit(ctx, ng, pos, delta)
    phi = torch.zeros_like(delta)
    prec = B.MG_PREC_FP64 if a.precision == "fp64" else B.MG_PREC_MIXED
    o = B.opts(rtol=a.rtol, precision=prec)
    inst = dict(ng=ng, box_mpch=a.box, a=1.0, omega_m=0.3, rc_h0=a.rc, delta=delta, phi=phi)

    for _ in range(a.warmup):
        B.mg_solve_dgp(ctx, [inst], o)
    torch.cuda.synchronize(dev)

    ctx.set_profiling(True)
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    stats = []
    for _ in range(a.steps):
        rcode, st = B.mg_solve_dgp(ctx, [inst], o)
        stats.append(st[0])
    e1.record()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ctx.set_profiling(False)
    ms = e0.elapsed_time(e1)
    updates = sum(s.cell_updates for s in stats)
    launches = sum(s.kernel_launches for s in stats)
    fs_ms = sum(s.fine_smooth_ms for s in stats)
    fs_n = sum(s.fine_smooth_launches for s in stats)
    t = torch.tensor([ms, float(updates)], dtype=torch.float64, device=dev)
    if dist:
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm_ = t.clone()
        dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
        ms_max, upd_tot = float(mx[0]), float(sm_[1])
    else:
        ms_max, upd_tot = ms, float(updates)
    value = upd_tot / (ms_max * 1e-3) / 1e9

    # end to end through the same C-ABI call with host buffers (pinned):
    # H2D of delta and D2H of phi inside the timed region
    e2e = None
    if not a.no_e2e:
        dh = delta.cpu().pin_memory()
        ph = torch.zeros_like(dh).pin_memory()
        insth = dict(inst, delta=dh, phi=ph)
        B.mg_solve_dgp(ctx, [insth], o)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        upd = 0
        for _ in range(a.steps):
            _, st = B.mg_solve_dgp(ctx, [insth], o)
            upd += st[0].cell_updates
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt, float(upd)], dtype=torch.float64, device=dev)
        if dist:
            mx = tt.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            sm_ = tt.clone()
            dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
            dt, upd = float(mx[0]), float(sm_[1])
        e2e = {"value": upd / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * ng ** 3,
               "d2h_bytes_per_step": 8 * ng ** 3}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    st0 = stats[-1]
    hbm_peak, peak_src = peaks()
    fp64_tf, fp32_tf = ctx.probe_alu_peaks()
    avg_launch_ms = fs_ms / max(fs_n, 1)
    # dominant kernel: the finest-level half-sweep (K1).  Algorithmic bytes per
    # launch: read both colour arrays, read the source of the updated colour,
    # write the updated colour = 2 s ng^3 (s = 8 bytes FP64, 4 FP32).
    s_bytes = 8 if a.precision == "fp64" else 4
    alg_bytes = 2 * s_bytes * ng ** 3
    achieved_gbs = alg_bytes / (avg_launch_ms * 1e-3) / 1e9
    # algorithmic FP64 operations per cell of the nDGP half-sweep (sqrt and
    # divide counted once each, an FMA as two)
    flops_cell = 44
    cells = ng ** 3 / 2
    achieved_tf = flops_cell * cells / (avg_launch_ms * 1e-3) / 1e12
    if a.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_tf, "traffic": None,
                "kernel": "k_smooth<double> finest half-sweep",
                "peak_source": "FP64 FMA rate measured by mg_probe_alu_peaks on this GPU",
                "hbm_view": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_source": peak_src},
                "avg_launch_ms": avg_launch_ms, "launches": fs_n, "alg_bytes_per_launch": alg_bytes,
                "alg_flops_per_cell": flops_cell}
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": None, "kernel": "k_smooth<float> finest half-sweep",
                "peak_source": peak_src, "avg_launch_ms": avg_launch_ms, "launches": fs_n,
                "alg_bytes_per_launch": alg_bytes}
    cb = None
    if not a.no_cpu:
        cb = cpu_baseline(delta.cpu().numpy(), a)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "nDGP FAS V(2,2) solve to eps/eps_ref<%g, %d^3 mesh, CIC of %d^3 Zel'dovich "
                                   "particles (P~k^0.96 e^-k/5, sigma8=0.8, z=0), L=%g Mpc/h, a=1, Omega_m=0.3, "
                                   "H0 rc=%g" % (a.rtol, ng, a.np, a.box, a.rc),
                       "precision": a.precision, "cycles_per_solve": st0.cycles,
                       "cell_updates_per_solve": st0.cell_updates,
                       "l2": "inputs larger than L2 (delta %d MB, phi %d MB)" % (8 * ng ** 3 >> 20, 8 * ng ** 3 >> 20),
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "gpu_launches": launches,
            "clocks": ck,
            "roofline": roof,
            "alu_peaks_tflops": {"fp64": fp64_tf, "fp32": fp32_tf},
            "e2e": e2e,
            "cpu_baseline": cb}
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
