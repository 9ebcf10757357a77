#!/usr/bin/env python3
"""Benchmark of the hot path: the nDGP (Vainshtein) multigrid field solve of
MG-GLAM (arXiv:2110.00566, Sec. 3.2) on a 512^3 periodic mesh.

Workload (synthetic, seeded): the particle-mesh run of Sec. 3.1 that the
solve sits in -- 256^3 particles in a 256 Mpc/h box from Zel'dovich initial
conditions at z = 100 (P(k) = A k^0.96 exp(-k/5), sigma_8 = 0.8, seed 2 +
rank), 100 leapfrog steps of constant da to z = 0 on the 512^3 mesh with an
FP64 nDGP solve (H0 r_c = 1, warm-started) at every step -- and, as the
timed step, the nDGP solve of that run's z = 0 CIC density: a = 1,
Omega_m = 0.3, from phi = 0 to eps/eps_ref < 1e-8 with V(2,2) cycles
(source prep, all cycles, gauge fix), inputs resident in HBM.  The metric
is smoother cell-updates (summed over all levels and cycles) per second.

`value` is the FP64 solve (every level FP64, the paper's precision).  The
same line reports the forms under "forms" (mixed precision, the batched
ensemble, the adjoint, the 100-step run itself at H0 r_c = 1 and 5, the
Kmouflage solves, the cycle types) and a compact "forms_summary" as its
last key.

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
# algorithmic FP64 operations per cell of the nDGP half-sweep (sqrt counted
# once, an FMA as two): S_a, their differences and C_ab (3 + 3 + 9 adds),
# the two sums of squares (2 x 5), Q (3), Sigma (1), the sqrt argument (2),
# sqrt (1), N (2), the face sum (2), N + f - c (2), the update (3) = 41
FLOPS_PER_CELL_FP64 = 41
# Thread instructions per updated cell of the FP64 nDGP half-sweep
# (k_smooth_bfp, the finest level: stencil staged in shared memory as block
# fixed point, sums and quadratic form on the integer pipes), from ncu's
# sm__inst_executed_pipe_{fp64,alu,fmaheavy} and sm__inst_executed counters
# at 256^3 (profiles/k_smooth_bfp_fp64_ndgp_256.md), and what each pipe
# issues per SM per clock: ALU and the FMA pipe's integer half 4
# sub-partitions x 16 lanes, all instructions 4 x 32; the FP64 rate comes
# from the probe at run time
FP64_MIX = {"fp64": 5.0, "alu": 259.0, "fma": 122.0, "issue": 522.0}
PIPE_RATE = {"alu": 64.0, "fma": 64.0, "issue": 128.0}


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
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--forms", default="all",
                   help="comma-separated forms to run: mixed, accuracy, rc5, batched, adjoint, adjoint_pm, "
                        "kmouflage, cycles (default all; --no-forms runs none)")
    p.add_argument("--inner", type=int, default=0, help="FP32 cycles per FP64 defect (0: library default)")
    p.add_argument("--fp32-smoother", type=int, default=0,
                   help="FP32 half-sweep kernel: 0 autotuned, -1 gathering, k >= 1 streaming variant k")
    p.add_argument("--fp32-shape", default="",
                   help="pin the gathering FP32 half-sweep shape, n:bx:zc[,n:bx:zc...] (profiling)")
    p.add_argument("--batch", type=int, default=64, help="instances of the batched form (0: skip)")
    p.add_argument("--adj-ng", type=int, default=128, help="mesh of the adjoint form (0: skip)")
    p.add_argument("--pm-adj-ng", type=int, default=128,
                   help="mesh (= particles per side) of the differentiable PM run (0: skip)")
    p.add_argument("--pm-adj-steps", type=int, default=20)
    p.add_argument("--fd-dirs", type=int, default=16, help="finite-difference directions for the PM gradient")
    p.add_argument("--pm-steps", type=int, default=100,
                   help="leapfrog steps of the particle-mesh run whose z = 0 density is the solve's input "
                        "(0: the Zel'dovich field at z = 0 instead)")
    p.add_argument("--cpu-full-ng", type=int, default=256,
                   help="mesh of the oracle's complete solve in the CPU baseline (0: skip)")
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
    levels = oracle.num_levels(ng)
    for l in range(levels):
        cells = (ng >> l) ** 3
        per_cycle += (oracle.Opts().coarse_sweeps if l == levels - 1 else 4) * cells
    updates = per_cycle * st.cycles
    out = {"value": updates / dt / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "%d V(2,2) cycle(s) of the %d^3 solve (with its initial and final residual passes), "
                     "plain C FP64 oracle, OpenMP over i-planes" % (st.cycles, ng),
           "seconds": dt}
    if getattr(a, "cpu_full_ng", 0) > 0:
        out["full_solve"] = cpu_full_solve(a.cpu_full_ng, a)
    return out


def cpu_full_solve(n, a):
    """The oracle's complete solve to eps/eps_ref < rtol on a smaller mesh of
    the same resolution (n^3 cells, (n/2)^3 Zel'dovich particles at z = 0,
    L = n/2 Mpc/h, seed 2): the CPU time of a whole solve, not a sample."""
    import oracle
    from paper_2110_00566_gb300 import inputs
    pos, _ = inputs.zeldovich(n // 2, n, n / 2.0, inputs.pk_cutoff(0.96, 5.0, 0.8), 1.0, seed=2)
    delta, _ = oracle.cic_deposit(pos, n, n // 2)
    t = time.perf_counter()
    u, st = oracle.dgp_solve(delta, 1.0, 0.3, a.rc, oracle.Opts(rtol=a.rtol, max_cycles=60))
    dt = time.perf_counter() - t
    levels = oracle.num_levels(n)
    per_cycle = sum((oracle.Opts().coarse_sweeps if l == levels - 1 else 4) * (n >> l) ** 3 for l in range(levels))
    return {"value": per_cycle * st.cycles / dt / 1e9, "unit": UNIT, "ms_per_solve": dt * 1e3,
            "cycles": st.cycles, "cores": os.cpu_count(),
            "sample": "complete FP64 solve to eps/eps_ref < %g of a %d^3 mesh (CIC of %d^3 Zel'dovich particles "
                      "at z = 0, L = %g Mpc/h), plain C oracle, OpenMP over i-planes" % (a.rtol, n, n // 2, n / 2.0)}


def summarise(line, primary):
    """A compact digest of the forms, the line's last key: each form as a
    speedup over the plain FP64 GPU solve (the headline), with the numbers
    it rests on."""
    f = line.get("forms", {})

    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d

    out = {"fp64_ms": round(primary["ms_per_step"], 2), "fp64_hbm_frac": g(line, "roofline", "frac"),
           "mixed_ms": g(f, "mixed", "ms_per_step"), "mixed_speedup_at_rtol": g(f, "mixed", "speedup_vs_primary"),
           "mixed_hbm_frac": g(f, "mixed", "roofline", "frac"),
           "at_1e-6_fp64_ms": g(f, "at_equal_accuracy", "fp64", "ms"),
           "at_1e-6_mixed_ms": g(f, "at_equal_accuracy", "mixed", "ms"),
           "at_1e-6_mixed_speedup": g(f, "at_equal_accuracy", "mixed_speedup"),
           "batched_ms": g(f, "batched", "ms_per_batch"),
           "batched_speedup_vs_fp64_loop": g(f, "batched", "speedup_vs_fp64_loop"),
           "batched_speedup_vs_mixed_loop": g(f, "batched", "speedup_vs_sequential"),
           "batched_at_1e-6_speedup_vs_fp64_loop": g(f, "batched", "at_equal_accuracy", "speedup_vs_fp64_loop"),
           "adjoint_backward_over_forward": g(f, "adjoint", "backward_over_forward"),
           "adjoint_pm_reverse_over_forward": g(f, "adjoint_pm", "reverse_over_forward"),
           "pm100_rc1_ms_per_step": g(f, "pm_run", "rc1", "ms_per_step"),
           "pm100_rc1_solve_share": g(f, "pm_run", "rc1", "solve_share"),
           "pm100_rc1_cycles_per_step": g(f, "pm_run", "rc1", "cycles_per_step_mean"),
           "pm100_rc5_ms_per_step": g(f, "pm_run", "rc5", "ms_per_step"),
           "rc5_fp64_ms": g(f, "rc5", "fp64", "ms_per_solve"), "rc5_mixed_ms": g(f, "rc5", "mixed", "ms_per_solve"),
           "kmo_n2_fp64_ms": g(f, "kmouflage", "n2_K0_1", "fp64", "ms"),
           "kmo_n2_mixed_ms": g(f, "kmouflage", "n2_K0_1", "mixed", "ms"),
           "kmo_n3_fp64_ms": g(f, "kmouflage", "n3_K0_1", "fp64", "ms"),
           "kmo_n3_mixed_ms": g(f, "kmouflage", "n3_K0_1", "mixed", "ms"),
           "cpu_full_solve_ms": g(line, "cpu_baseline", "full_solve", "ms_per_solve")}
    return {k: v for k, v in out.items() if v is not None}


def reduce_over_ranks(dist, ms, updates, device):
    """Whole-job numbers of a replicas run: the slowest rank's time (max) and
    the updates of all ranks (sum); the identity without a process group."""
    import torch
    if not dist:
        return ms, float(updates)
    mx = torch.tensor([ms], dtype=torch.float64, device=device)
    sm = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


def workload_name(a):
    if getattr(a, "pm_steps", 0) > 0:
        src = ("z=0 CIC density of a %d-step PM run of %d^3 particles (Zel'dovich ICs at z=100, "
               "P~k^0.96 e^-k/5, sigma8=0.8, nDGP solve every step)" % (a.pm_steps, a.np))
    else:
        src = "CIC of %d^3 Zel'dovich particles (P~k^0.96 e^-k/5, sigma8=0.8, z=0)" % a.np
    return ("nDGP FAS V(2,2) solve to eps/eps_ref<%g, %d^3 mesh, %s, L=%g Mpc/h, a=1, Omega_m=0.3, H0 rc=%g"
            % (a.rtol, a.ng, src, a.box, a.rc))


def run_reference(a, rank, world):
    if rank != 0:
        return
    a.cpu_full_ng = 0   # each step is the bounded one-cycle sample only
    import numpy as np
    import oracle
    pos = particles(a, 0)
    delta, _ = oracle.cic_deposit(pos, a.ng, a.np)
    vals = []
    for _ in range(a.warmup):
        cpu_baseline(delta, a)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        cb = cpu_baseline(delta, a)
        vals.append(cb["value"])
    dt = time.perf_counter() - t0
    v = float(np.mean(vals))
    cb["value"] = v
    if a.pm_steps > 0:
        cb["sample"] += ("; input: the Zel'dovich density at z = 0 of the same initial conditions (the "
                         "%d-step particle-mesh run that evolves them is not part of the sample)" % a.pm_steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(a), "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        from oracle import build as ob
        ob.build()
        return run_reference(a, rank, world)

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
    if a.fp32_smoother:
        ctx.set_fp32_smoother(a.fp32_smoother)
    for item in filter(None, a.fp32_shape.split(",")):
        ctx.set_fp32_smoother_shape(*(int(x) for x in item.split(":")))
    ng = a.ng
    # the end-to-end call's pinned host buffers, taken before the run's
    # large host allocations (so that they do not land on fragmented pages)
    pinned = None if a.no_e2e else [torch.empty((ng,) * 3, dtype=torch.float64).pin_memory() for _ in range(2)]

    def pm_run(rc, model=1, box=None):
        """The particle-mesh run of the workload (Sec. 3.1 and 3.1.1): a.np^3
        particles on the ng^3 mesh in a box of L Mpc/h, Zel'dovich initial
        conditions at z = 100 on the growing mode (x = q + D psi,
        p = a^2 E D f psi; seed 2 + rank), a.pm_steps leapfrog steps of
        constant da to a = 1 (the first a half kick), FP32 particle state and,
        for model 1, the FP64 nDGP solve (H0 r_c = rc, Sec. 3.2.3) at every
        step to eps/eps_ref < rtol, warm-started from the previous step's
        field.  Returns the z = 0 positions and the run's timings."""
        import numpy as np
        from paper_2110_00566_gb300 import inputs
        box = box or a.box
        a0, om = 1.0 / 101.0, 0.3
        D, f = inputs.growth_lcdm(a0, om), inputs.growth_rate_lcdm(a0, om)
        E0 = float(np.sqrt(om / a0 ** 3 + 1.0 - om))
        p_, m_ = inputs.zeldovich(a.np, ng, box, inputs.pk_cutoff(0.96, 5.0, 0.8), D, seed=2 + rank,
                                  vel_factor=a0 * a0 * E0 * f * D)
        pos = torch.from_numpy(p_).to(dev)
        mom = torch.from_numpy(m_).to(dev)
        phi_ws = torch.zeros((ng, ng, ng), dtype=torch.float64, device=dev) if model else None
        da = (1.0 - a0) / a.pm_steps
        st = B.make_pm_state(pos, mom, ng, box, om, a0, da, model=model, rc_h0=rc, first=True, phi_ws=phi_ws)
        o = B.opts(rtol=a.rtol, max_cycles=60)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cyc, solve_ms, warn = [], 0.0, 0
        for _ in range(a.pm_steps):
            rcode, sst = B.pm_step(ctx, st, o)
            warn += int(rcode != 0)
            if model:
                cyc.append(sst.cycles)
                solve_ms += sst.ms
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        res = {"steps": a.pm_steps, "particles": a.np ** 3, "ng": ng, "box_mpch": box, "z_start": 100.0,
               "a_end": st.a, "model": ["GR", "nDGP", "Kmouflage"][model], "ms_total": ms,
               "ms_per_step": ms / a.pm_steps, "precision": "FP32 particles" + (", FP64 solve" if model else "")}
        if model:
            res.update({"rc_h0": rc, "solve_ms_total": solve_ms, "solve_share": solve_ms / ms,
                        "cycles_per_step_mean": float(np.mean(cyc)), "cycles_per_step_max": int(max(cyc)),
                        "cycles_first_step": cyc[0], "steps_not_converged": warn,
                        "warm_start": "previous step's field"})
        return pos, res

    pm_forms = {}
    if a.pm_steps > 0:
        pos, pm_forms["rc%g" % a.rc] = pm_run(a.rc)
    else:
        pos = torch.from_numpy(particles(a, rank)).to(dev)
    delta = torch.empty((ng, ng, ng), dtype=torch.float64, device=dev)
    B.pm_cic_deposit(ctx, ng, pos, delta)
    del pos
    hbm_peak, peak_src = peaks()

    def reduce_max_sum(x, y):
        return reduce_over_ranks(dist, x, y, dev)

    def timed(precision):
        """W untimed + K timed solves; CUDA events on the caller's stream
        bracket the library's stream (ordered by events at entry/exit)."""
        prec = B.MG_PREC_FP64 if precision == "fp64" else B.MG_PREC_MIXED
        o = B.opts(rtol=a.rtol, precision=prec, max_cycles=60)
        if a.inner > 0:
            o.inner_cycles = a.inner
        phi = torch.zeros_like(delta)
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
            _, st = B.mg_solve_dgp(ctx, [inst], o)
            stats.append(st[0])
        e1.record()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        ck = clocks.stop()
        ctx.set_profiling(False)
        ms, upd = reduce_max_sum(e0.elapsed_time(e1), sum(s.cell_updates for s in stats))
        r = {"value": upd / (ms * 1e-3) / 1e9, "ms_per_step": ms / a.steps, "clocks": ck, "stats": stats,
             "phi": phi, "inst": inst, "o": o,
             "launches": sum(s.kernel_launches for s in stats),
             "avg_launch_ms": sum(s.fine_smooth_ms for s in stats) / max(1, sum(s.fine_smooth_launches for s in stats)),
             "fine_launches": sum(s.fine_smooth_launches for s in stats)}
        return r

    def e2e(r):
        """Same call with pinned host buffers: H2D of delta and D2H of phi
        inside the timed region."""
        dh, ph = pinned
        dh.copy_(delta)
        ph.zero_()
        insth = dict(r["inst"], delta=dh, phi=ph)
        B.mg_solve_dgp(ctx, [insth], r["o"])
        if dist:
            dist.barrier()
        clocks = Clocks(local)
        clocks.start()
        t0 = time.perf_counter()
        upd, solve_ms = 0, 0.0
        for _ in range(a.steps):
            _, st = B.mg_solve_dgp(ctx, [insth], r["o"])
            upd += st[0].cell_updates
            solve_ms += st[0].ms
        wall = time.perf_counter() - t0
        dt, upd = reduce_max_sum(wall, upd)
        # the library's own device time of each solve (events around the
        # solve on its stream, copies excluded) beside the wall time per call
        return {"value": upd / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * ng ** 3,
                "d2h_bytes_per_step": 8 * ng ** 3, "ms_per_step": 1e3 * wall / a.steps,
                "solve_ms_per_step": solve_ms / a.steps,
                "host_copy_gbs": 2 * 8 * ng ** 3 / max(1e-9, wall / a.steps - 1e-3 * solve_ms / a.steps) / 1e9,
                "clocks": clocks.stop()}

    # DRAM bytes (read + write) per launch of the dominant kernels from ncu,
    # with the mesh they were measured on (profiles/k_smooth_bfp_fp64_ndgp_256.md
    # and profiles/k_smooth4_fp32corr_ndgp_512.md, both at 512^3), scaled by
    # the cell count to this mesh
    TRAFFIC = {"fp64": (1676.4e6 + 515.9e6, 512), "mixed": (1670.8e6 + 255.4e6, 512)}

    def roofline(r, precision, fp64_tf):
        """Roofline of the finest half-sweep, anchored to the HBM peak (the
        metric's "% of HBM peak"): achieved = the algorithmic bytes of one
        launch over its average CUDA-event duration in the timed solves."""
        ms = r["avg_launch_ms"]
        tb, tn = TRAFFIC[precision]
        traffic = tb * (ng / float(tn)) ** 3
        tsrc = "ncu dram__bytes_read.sum + dram__bytes_write.sum at %d^3%s" % (
            tn, "" if tn == ng else ", scaled by (ng/%d)^3" % tn)
        if precision == "fp64":
            # finest FP64 half-sweep: read both colours + the colour's s,
            # write the colour = 2 s n^3 bytes (s = 8).  Its limiter is the
            # arithmetic pipes, not HBM: the instruction-mix speed of light
            # (the busiest pipe's issue time at the sampled SM clock) and the
            # algorithmic FP64 flops against the FP64 FMA rate are reported
            # beside the HBM fraction as diagnostics
            cells = ng ** 3 / 2
            alg = 2 * 8 * ng ** 3
            gbs = alg / (ms * 1e-3) / 1e9
            tf = FLOPS_PER_CELL_FP64 * cells / (ms * 1e-3) / 1e12
            mhz = (r.get("clocks") or {}).get("sm_mhz") or 2070.0
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            rate64 = fp64_tf * 1e12 / 2.0 / (nsm * mhz * 1e6)   # FP64 instructions per clock per SM
            cyc = {"fp64": FP64_MIX["fp64"] / rate64, "alu": FP64_MIX["alu"] / PIPE_RATE["alu"],
                   "fma": FP64_MIX["fma"] / PIPE_RATE["fma"], "issue": FP64_MIX["issue"] / PIPE_RATE["issue"]}
            bind = max(cyc, key=cyc.get)
            t_sol = cells / nsm * cyc[bind] / (mhz * 1e6)
            return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "traffic": traffic, "traffic_source": tsrc, "kernel": "k_smooth_bfp finest half-sweep",
                    "peak_source": peak_src + " HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "alg_bytes_per_launch": alg, "avg_launch_ms": ms, "launches": r["fine_launches"],
                    "limiter": "integer ALU and FP64 issue (instruction mix), not HBM",
                    "alu_view": {"achieved": tf, "unit": "TFLOP/s", "alg_flops_per_cell": FLOPS_PER_CELL_FP64,
                                 "fp64_fma_peak": fp64_tf, "frac_of_fp64_fma_peak": tf / fp64_tf,
                                 "instruction_mix_sol_ms": t_sol * 1e3, "frac_of_instruction_mix_sol": t_sol * 1e3 / ms,
                                 "binding_pipe": bind, "instructions_per_cell": FP64_MIX,
                                 "sm_clocks_per_cell": cyc, "sm_mhz": mhz}}
        # finest FP32 correction half-sweep: read e and the base field (both
        # colours, 4 B each), s and f of the colour (2 B each), write the
        # colour (2 B) = 14 n^3 bytes
        alg = 14 * ng ** 3
        gbs = alg / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": traffic, "traffic_source": tsrc, "kernel": "k_smooth4<float, correction, nDGP> finest half-sweep",
                "peak_source": peak_src, "avg_launch_ms": ms, "launches": r["fine_launches"],
                "alg_bytes_per_launch": alg}

    def at_accuracy(dl, rc, tol=1e-6):
        """The FP64 and mixed-precision solves at the same accuracy: the
        loosest rtol in {1e-4 ... 1e-8} whose phi lies within tol (relative
        L2) of a tight FP64 solution (rtol 1e-12), each timed over a.steps
        solves from phi = 0."""
        inst = dict(ng=ng, box_mpch=a.box, a=1.0, omega_m=0.3, rc_h0=rc, delta=dl)
        ref = torch.zeros_like(dl)
        B.mg_solve_dgp(ctx, [dict(inst, phi=ref)], B.opts(rtol=1e-12, max_cycles=60))
        nref = torch.linalg.vector_norm(ref)
        out = {"tolerance": tol, "reference": "FP64 solve to eps/eps_ref < 1e-12"}
        for name, prec in (("fp64", B.MG_PREC_FP64), ("mixed", B.MG_PREC_MIXED)):
            phi = torch.zeros_like(dl)
            pick = None
            for rt in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
                o = B.opts(rtol=rt, precision=prec, max_cycles=60)
                phi.zero_()
                B.mg_solve_dgp(ctx, [dict(inst, phi=phi)], o)
                err = float(torch.linalg.vector_norm(phi - ref) / nref)
                if err <= tol:
                    pick = (rt, err, o)
                    break
            if pick is None:
                out[name] = {"reached": False}
                continue
            rt, err, o = pick
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cyc = 0
            for _ in range(a.steps):
                _, st = B.mg_solve_dgp(ctx, [dict(inst, phi=phi)], o)
                cyc = st[0].cycles
            e1.record()
            torch.cuda.synchronize(dev)
            out[name] = {"rtol": rt, "phi_rel_l2_vs_tight": err, "ms": e0.elapsed_time(e1) / a.steps,
                         "cycles": cyc}
        if "ms" in out.get("fp64", {}) and "ms" in out.get("mixed", {}):
            out["mixed_speedup"] = out["fp64"]["ms"] / out["mixed"]["ms"]
        return out

    def batched():
        """Emulator ensemble: a.batch independent solves, N uniform over
        {64, 96, 128, 192, 256}, L = N Mpc/h, N/2 particles per side,
        Zel'dovich at z = 0 with sigma_8 ~ U[0.7, 0.9], H0 r_c log-uniform in
        [0.5, 10] (seed 4 + rank); mixed precision.  The batched call (one
        persistent kernel) against a loop of single mixed-precision solves
        and against a loop of plain FP64 solves (the FP64 GPU baseline of the
        forms), with the batched phi's distance to the FP64 loop's."""
        import numpy as np
        from paper_2110_00566_gb300 import inputs
        rng = np.random.default_rng(4 + rank)
        insts, seq = [], []
        for q in range(a.batch):
            n = int(rng.choice([64, 96, 128, 192, 256]))
            sig8 = float(rng.uniform(0.7, 0.9))
            rc = float(np.exp(rng.uniform(np.log(0.5), np.log(10.0))))
            p_, _ = inputs.zeldovich(n // 2, n, float(n), inputs.pk_cutoff(sigma8=sig8), 1.0, seed=100 + q)
            d = torch.empty((n, n, n), dtype=torch.float64, device=dev)
            B.pm_cic_deposit(ctx, n, torch.from_numpy(p_).to(dev), d)
            insts.append(dict(ng=n, box_mpch=float(n), a=1.0, omega_m=0.3, rc_h0=rc, delta=d,
                              phi=torch.zeros_like(d)))
            seq.append(dict(insts[-1], phi=torch.zeros_like(d)))
        o = B.opts(rtol=a.rtol, precision=B.MG_PREC_MIXED, max_cycles=60)
        if a.inner > 0:
            o.inner_cycles = a.inner
        for _ in range(max(1, a.warmup)):
            B.mg_solve_dgp(ctx, insts, o)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        upd = 0
        for _ in range(a.steps):
            _, st = B.mg_solve_dgp(ctx, insts, o)
            upd += sum(s.cell_updates for s in st)
        e1.record()
        torch.cuda.synchronize(dev)
        ms_b = e0.elapsed_time(e1) / a.steps
        for inst in seq:
            B.mg_solve_dgp(ctx, [inst], o)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(a.steps):
            for inst in seq:
                B.mg_solve_dgp(ctx, [inst], o)
        e1.record()
        torch.cuda.synchronize(dev)
        ms_s = e0.elapsed_time(e1) / a.steps
        worst = max(float(torch.linalg.vector_norm(x["phi"] - y["phi"]) / torch.linalg.vector_norm(y["phi"]))
                    for x, y in zip(insts, seq))
        # the plain FP64 loop (one timed pass: it is the slow baseline)
        o64 = B.opts(rtol=a.rtol, precision=B.MG_PREC_FP64, max_cycles=60)
        seq64 = [dict(x, phi=torch.zeros_like(x["delta"])) for x in insts]
        for inst in seq64[:8]:
            B.mg_solve_dgp(ctx, [dict(inst, phi=torch.zeros_like(inst["delta"]))], o64)
        torch.cuda.synchronize(dev)
        e0.record()
        for inst in seq64:
            B.mg_solve_dgp(ctx, [inst], o64)
        e1.record()
        torch.cuda.synchronize(dev)
        ms_64 = e0.elapsed_time(e1)
        worst64 = max(float(torch.linalg.vector_norm(x["phi"] - y["phi"]) / torch.linalg.vector_norm(y["phi"]))
                      for x, y in zip(insts, seq64))
        cells = sum(x["ng"] ** 3 for x in insts)
        # at the same accuracy: the loosest rtol at which every instance's phi
        # lies within 1e-6 (relative L2) of its tight FP64 solution, for the
        # batched call and for the loop of plain FP64 solves
        tight = [torch.zeros_like(x["delta"]) for x in insts]
        for x, t in zip(insts, tight):
            B.mg_solve_dgp(ctx, [dict(x, phi=t)], B.opts(rtol=1e-12, max_cycles=60))

        def worst_vs_tight(phis):
            return max(float(torch.linalg.vector_norm(p - t) / torch.linalg.vector_norm(t))
                       for p, t in zip(phis, tight))

        acc = {"tolerance": 1e-6}
        for rt in (1e-5, 1e-6, 1e-7, 1e-8):
            ob = B.opts(rtol=rt, precision=B.MG_PREC_MIXED, max_cycles=60)
            B.mg_solve_dgp(ctx, insts, ob)
            wb = worst_vs_tight([x["phi"] for x in insts])
            if wb <= 1e-6:
                torch.cuda.synchronize(dev)
                e0.record()
                B.mg_solve_dgp(ctx, insts, ob)
                e1.record()
                torch.cuda.synchronize(dev)
                acc["batched"] = {"rtol": rt, "ms": e0.elapsed_time(e1), "phi_worst_rel_l2_vs_tight": wb}
                break
        for rt in (1e-5, 1e-6, 1e-7, 1e-8):
            o64r = B.opts(rtol=rt, precision=B.MG_PREC_FP64, max_cycles=60)
            torch.cuda.synchronize(dev)
            e0.record()
            for inst in seq64:
                B.mg_solve_dgp(ctx, [inst], o64r)
            e1.record()
            torch.cuda.synchronize(dev)
            w64 = worst_vs_tight([x["phi"] for x in seq64])
            if w64 <= 1e-6:
                acc["fp64_loop"] = {"rtol": rt, "ms": e0.elapsed_time(e1), "phi_worst_rel_l2_vs_tight": w64}
                break
        if "batched" in acc and "fp64_loop" in acc:
            acc["speedup_vs_fp64_loop"] = acc["fp64_loop"]["ms"] / acc["batched"]["ms"]
        return {"value": upd / a.steps / (ms_b * 1e-3) / 1e9, "unit": UNIT, "instances": a.batch,
                "total_cells": cells, "ms_per_batch": ms_b, "ms_sequential_loop": ms_s,
                "speedup_vs_sequential": ms_s / ms_b, "phi_rel_l2_vs_sequential_max": worst,
                "ms_fp64_loop": ms_64, "speedup_vs_fp64_loop": ms_64 / ms_b, "phi_rel_l2_vs_fp64_max": worst64,
                "sizes": sorted({x["ng"] for x in insts}), "launch": "one persistent cooperative kernel, graph-captured",
                "at_equal_accuracy": acc}

    def adjoint():
        """Backward/forward: the FP64 adjoint solve (mg_solve_adjoint) vs the
        FP64 forward solve at a.adj_ng^3 (CIC of a Zel'dovich load, L = 2 N)."""
        import numpy as np
        from paper_2110_00566_gb300 import inputs
        n = a.adj_ng
        p_, _ = inputs.zeldovich(n, n, 2.0 * n, inputs.pk_cutoff(), 1.0, seed=5)
        d = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        B.pm_cic_deposit(ctx, n, torch.from_numpy(p_).to(dev), d)
        phi = torch.zeros_like(d)
        g = torch.from_numpy(inputs.white_noise(n, 6)).to(dev)
        out = torch.empty_like(d)
        o = B.opts(rtol=a.rtol, max_cycles=60)
        inst = dict(ng=n, box_mpch=2.0 * n, a=1.0, omega_m=0.3, rc_h0=a.rc, delta=d, phi=phi)
        for _ in range(2):
            B.mg_solve_dgp(ctx, [inst], o)
            B.mg_solve_adjoint(ctx, n, 2.0 * n, 1.0, 0.3, a.rc, phi, d, g, out, o)
        torch.cuda.synchronize(dev)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        for _ in range(a.steps):
            B.mg_solve_dgp(ctx, [inst], o)
        e1.record()
        cyc = 0
        for _ in range(a.steps):
            _, _, st = B.mg_solve_adjoint(ctx, n, 2.0 * n, 1.0, 0.3, a.rc, phi, d, g, out, o)
            cyc = st.cycles
        e2.record()
        torch.cuda.synchronize(dev)
        fwd, bwd = e0.elapsed_time(e1) / a.steps, e1.elapsed_time(e2) / a.steps
        return {"ng": n, "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
                "adjoint_cycles": cyc, "precision": "fp64"}

    def kmouflage(pos_z0=None):
        """Kmouflage solves on the headline mesh with a 512 Mpc/h box: the
        z = 0 density of the same seeded run in that box (GR dynamics), or
        without a run the Zel'dovich load at z = 0 (seed 3); (n, K0) =
        (2, 1) and (3, 1), beta = 0.2, a = 1, with lambda, phibar'/H0 and
        A(phibar) from the library's background solve of each model; the
        FP64 solve and the mixed-precision solve, the latter's phi against
        the former's (both to rtol)."""
        import numpy as np
        from paper_2110_00566_gb300 import inputs
        box = 2.0 * a.box
        if pos_z0 is None:
            pk = inputs.pk_cutoff(0.96, 5.0, 0.8)
            p_, _ = inputs.zeldovich(a.np, ng, box, pk, 1.0, seed=3)
            pos_z0 = torch.from_numpy(p_).to(dev)
        dk = torch.empty((ng, ng, ng), dtype=torch.float64, device=dev)
        B.pm_cic_deposit(ctx, ng, pos_z0, dk)
        out = {}
        for nk, k0 in ((2, 1.0), (3, 1.0)):
            t0 = time.perf_counter()
            _, lam, bgt = B.mg_kmo_background(B.kmo_background_params(n=nk, k0=k0, beta_kmo=0.2, omega_m=0.3), [1.0])
            bg_ms = (time.perf_counter() - t0) * 1e3
            dphi_h0, A_bar = float(bgt[0, 4]), float(bgt[0, 3])
            res = {}
            phis = {}
            for prec in ("fp64", "mixed"):
                o = B.opts(rtol=a.rtol, max_cycles=60,
                           precision=B.MG_PREC_FP64 if prec == "fp64" else B.MG_PREC_MIXED)
                phi = torch.zeros_like(dk)
                B.mg_solve_kmouflage(ctx, ng, box, 1.0, 0.3, nk, k0, 0.2, lam, dphi_h0, A_bar, dk, phi, o)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                _, st = B.mg_solve_kmouflage(ctx, ng, box, 1.0, 0.3, nk, k0, 0.2, lam, dphi_h0, A_bar, dk, phi, o)
                e1.record()
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1)
                res[prec] = {"ms": ms, "cycles": st.cycles, "value": st.cell_updates / (ms * 1e-3) / 1e9,
                             "final_eps_over_eps_ref": st.eps[st.n_eps - 1] / st.eps_ref}
                phis[prec] = phi
            l2 = float(torch.linalg.vector_norm(phis["mixed"] - phis["fp64"]) / torch.linalg.vector_norm(phis["fp64"]))
            # screening off: the linear-theory field (FFT), and the rms
            # gradient (fifth force) of the full field relative to it
            lin = torch.empty_like(dk)
            args = (ng, box, 1.0, 0.3, nk, k0, 0.2, lam, dphi_h0, A_bar)
            B.mg_solve_kmouflage_linear(ctx, *args, dk, lin)
            torch.cuda.synchronize(dev)
            e0.record()
            B.mg_solve_kmouflage_linear(ctx, *args, dk, lin)
            e1.record()
            torch.cuda.synchronize(dev)

            def grad_rms(f):
                g = [torch.roll(f, -1, d) - torch.roll(f, 1, d) for d in range(3)]
                return float(torch.sqrt(sum((x * x).mean() for x in g)))

            out["n%d_K0_%g" % (nk, k0)] = {"background": {"lambda": lam, "phibar_prime_over_h0": dphi_h0,
                                                          "A_bar": A_bar, "phibar": float(bgt[0, 1]),
                                                          "host_ms": bg_ms},
                                          "fp64": res["fp64"], "mixed": res["mixed"],
                                          "mixed_speedup": res["fp64"]["ms"] / res["mixed"]["ms"],
                                          "phi_rel_l2_mixed_vs_fp64": l2, "unit": UNIT,
                                          "linear_ms": e0.elapsed_time(e1),
                                          "fifth_force_rms_full_over_linear": grad_rms(phis["fp64"]) / grad_rms(lin)}
        out["config"] = "512^3 mesh, L = %g Mpc/h, beta = 0.2, a = 1" % box
        return out

    def cycle_types():
        """V-, F- and W-cycles on the headline solve (FP64, rtol as the
        headline): time, cycles and phi's distance to a tight reference
        (V-cycles to 1e-12), the error-versus-cost comparison of the cycle
        types."""
        ref = torch.zeros_like(delta)
        inst = dict(ng=ng, box_mpch=a.box, a=1.0, omega_m=0.3, rc_h0=a.rc, delta=delta)
        B.mg_solve_dgp(ctx, [dict(inst, phi=ref)], B.opts(rtol=1e-12, max_cycles=60))
        out = {}
        for name, cyc in (("V", B.MG_CYCLE_V), ("F", B.MG_CYCLE_F), ("W", B.MG_CYCLE_W)):
            o = B.opts(rtol=a.rtol, max_cycles=60, cycle=cyc)
            phi = torch.zeros_like(delta)
            B.mg_solve_dgp(ctx, [dict(inst, phi=phi)], o)
            phi.zero_()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = B.mg_solve_dgp(ctx, [dict(inst, phi=phi)], o)
            e1.record()
            torch.cuda.synchronize(dev)
            st = st[0]
            out[name] = {"ms": e0.elapsed_time(e1), "cycles": st.cycles,
                         "final_eps_over_eps_ref": st.eps[st.n_eps - 1] / st.eps_ref,
                         "phi_rel_l2_vs_tight": float(torch.linalg.vector_norm(phi - ref) / torch.linalg.vector_norm(ref))}
        out["precision"] = "fp64"
        return out

    def adjoint_pm():
        """The differentiable PM run of the adjoint workload: n^3 particles
        on an n^3 mesh, L = 2n Mpc/h, a.pm_adj_steps leapfrog steps from
        z = 10 to 0 with the nDGP solve (FP64) at every step, loss = MSE of
        the 32-bin P(k) against the spectrum of the run from another seed,
        gradients with respect to the white noise and R_c (checkpoints every
        4 steps).  Reports forward and forward+reverse times and the
        gradient against central differences along random unit directions."""
        import numpy as np
        from paper_2110_00566_gb300 import inputs
        n, box, a0 = a.pm_adj_ng, 2.0 * a.pm_adj_ng, 1.0 / 11.0
        D = inputs.growth_lcdm(a0, 0.3)
        E0 = float(np.sqrt(0.3 / a0 ** 3 + 0.7))
        cfg = B.make_dpm_config(n, box, 0.3, a0, 1.0, a.pm_adj_steps, 4, 32, 1, D,
                                a0 * a0 * E0 * D * inputs.growth_rate_lcdm(a0, 0.3))
        amp = torch.from_numpy(inputs.pk_amplitude(n, box, inputs.pk_cutoff())).to(dev)
        w = torch.from_numpy(inputs.white_noise(n, 5).astype(np.float32).astype(np.float64)).to(dev)
        w6 = torch.from_numpy(inputs.white_noise(n, 6).astype(np.float32).astype(np.float64)).to(dev)
        o = B.opts(rtol=1e-10, max_cycles=60)
        tgt, _, _, _ = B.dpm_run(ctx, cfg, amp, w6, a.rc, o=o)
        grad = torch.empty_like(w)
        B.dpm_run(ctx, cfg, amp, w, a.rc, tgt, grad, o=o)      # warm-up (workspace, plans)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, L0, _, stf = B.dpm_run(ctx, cfg, amp, w, a.rc, tgt, o=o)
        t1 = time.perf_counter()
        _, _, drc, stb = B.dpm_run(ctx, cfg, amp, w, a.rc, tgt, grad, o=o)
        t2 = time.perf_counter()
        fwd, both = (t1 - t0) * 1e3, (t2 - t1) * 1e3
        g = grad.cpu().numpy()
        errs = []
        eps = 1e-3
        for q in range(a.fd_dirs):
            v = inputs.white_noise(n, 700 + q)
            v /= np.linalg.norm(v)
            vt = torch.from_numpy(v).to(dev)
            lp = B.dpm_run(ctx, cfg, amp, w + eps * vt, a.rc, tgt, o=o)[1]
            lm = B.dpm_run(ctx, cfg, amp, w - eps * vt, a.rc, tgt, o=o)[1]
            fd = (lp - lm) / (2 * eps)
            ad = float(np.sum(g * v))
            errs.append(abs(ad - fd) / max(abs(fd), 1e-300))
        hr = 1e-4 * a.rc
        fdr = (B.dpm_run(ctx, cfg, amp, w, a.rc + hr, tgt, o=o)[1] - B.dpm_run(ctx, cfg, amp, w, a.rc - hr, tgt, o=o)[1]) / (2 * hr)
        return {"ng": n, "particles": n ** 3, "box_mpch": box, "steps": a.pm_adj_steps, "checkpoint_every": 4,
                "nbins": 32, "loss": L0, "forward_ms": fwd, "forward_and_reverse_ms": both,
                "reverse_over_forward": (both - fwd) / fwd, "solver_cycles_forward": stf.cycles,
                "solver_cycles_forward_and_reverse": stb.cycles,
                "fd_directions": a.fd_dirs, "fd_max_rel_err_noise": max(errs) if errs else None,
                "fd_median_rel_err_noise": float(np.median(errs)) if errs else None,
                "dL_dRc": drc, "fd_rel_err_Rc": abs(drc - fdr) / max(abs(fdr), 1e-300),
                "precision": "fp64 particles and solves"}

    names = set() if a.no_forms else (
        {"mixed", "accuracy", "rc5", "batched", "adjoint", "adjoint_pm", "kmouflage", "cycles"} if a.forms == "all"
        else set(x.strip() for x in a.forms.split(",") if x.strip()))

    def want(f):
        return f in names

    def ranged(name, fn, *args):
        """fn(*args) inside an NVTX range named for the form (profiling:
        ncu --nvtx --nvtx-include "<name>/")."""
        torch.cuda.nvtx.range_push(name)
        try:
            return fn(*args)
        finally:
            torch.cuda.nvtx.range_pop()

    primary = ranged("headline", timed, a.precision)
    # the end-to-end call right after the device-timed one, at the same
    # thermal state of the GPU (the forms that follow run it for minutes)
    e2e_primary = None if a.no_e2e else e2e(primary)
    second = None
    if want("mixed"):
        second = ranged("mixed", timed, "mixed" if a.precision == "fp64" else "fp64")
    acc_form = ranged("accuracy", at_accuracy, delta, a.rc) if want("accuracy") else None
    rc5_form = None
    if want("rc5") and a.pm_steps > 0 and a.rc != 5.0:
        # the run and the headline solve at H0 r_c = 5: its own z = 0 density
        pos5, pm_forms["rc5"] = pm_run(5.0)
        d5 = torch.empty_like(delta)
        B.pm_cic_deposit(ctx, ng, pos5, d5)
        del pos5
        rc5_form = {}
        for name, prec in (("fp64", B.MG_PREC_FP64), ("mixed", B.MG_PREC_MIXED)):
            o5 = B.opts(rtol=a.rtol, precision=prec, max_cycles=60)
            i5 = dict(ng=ng, box_mpch=a.box, a=1.0, omega_m=0.3, rc_h0=5.0, delta=d5, phi=torch.zeros_like(d5))
            B.mg_solve_dgp(ctx, [i5], o5)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            upd = 0
            for _ in range(a.steps):
                _, st5 = B.mg_solve_dgp(ctx, [i5], o5)
                upd += st5[0].cell_updates
            e1.record()
            torch.cuda.synchronize(dev)
            ms5 = e0.elapsed_time(e1)
            rc5_form[name] = {"value": upd / (ms5 * 1e-3) / 1e9, "unit": UNIT, "ms_per_solve": ms5 / a.steps,
                              "cycles": st5[0].cycles,
                              "final_eps_over_eps_ref": st5[0].eps[st5[0].n_eps - 1] / st5[0].eps_ref}
        del d5
    kmo_pos = None
    if want("kmouflage") and a.pm_steps > 0:
        kmo_pos, pm_forms["gr_512mpch"] = pm_run(0.0, model=0, box=2.0 * a.box)
    batch_form = ranged("batched", batched) if (a.batch > 0 and want("batched")) else None
    adj_form = ranged("adjoint", adjoint) if (a.adj_ng > 0 and want("adjoint")) else None
    pm_adj_form = ranged("adjoint_pm", adjoint_pm) if (a.pm_adj_ng > 0 and want("adjoint_pm")) else None
    kmo_form = ranged("kmouflage", kmouflage, kmo_pos) if want("kmouflage") else None
    kmo_pos = None
    cyc_form = ranged("cycles", cycle_types) if want("cycles") else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fp64_tf, fp32_tf = ctx.probe_alu_peaks()
    st0 = primary["stats"][-1]
    forms = {}
    if second is not None:
        name = "mixed" if a.precision == "fp64" else "fp64"
        st1 = second["stats"][-1]
        p0, p1 = primary["phi"], second["phi"]
        l2 = float(torch.linalg.vector_norm(p1 - p0) / torch.linalg.vector_norm(p0))
        forms[name] = {"value": second["value"], "unit": UNIT, "ms_per_step": second["ms_per_step"],
                       "speedup_vs_primary": primary["ms_per_step"] / second["ms_per_step"],
                       "phi_rel_l2_vs_primary": l2, "cycles_per_solve": st1.cycles,
                       "final_eps_over_eps_ref": st1.eps[st1.n_eps - 1] / st1.eps_ref,
                       "eps_measured_over_eps_ref": [st1.eps[q] / st1.eps_ref for q in range(st1.n_eps)],
                       "gpu_launches": second["launches"], "clocks": second["clocks"],
                       "roofline": roofline(second, name, fp64_tf)}
    if batch_form is not None:
        forms["batched"] = batch_form
    if adj_form is not None:
        forms["adjoint"] = adj_form
    if pm_adj_form is not None:
        forms["adjoint_pm"] = pm_adj_form
    if kmo_form is not None:
        forms["kmouflage"] = kmo_form
    if cyc_form is not None:
        forms["cycle_types"] = cyc_form
    if acc_form is not None:
        forms["at_equal_accuracy"] = acc_form
    if rc5_form is not None:
        forms["rc5"] = rc5_form
    if pm_forms:
        forms["pm_run"] = pm_forms
    cb = None if a.no_cpu else cpu_baseline(delta.cpu().numpy(), a)
    line = {"metric": METRIC, "value": primary["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": primary["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "precision": a.precision, "cycles_per_solve": st0.cycles,
                       "cell_updates_per_solve": st0.cell_updates,
                       "final_eps_over_eps_ref": st0.eps[st0.n_eps - 1] / st0.eps_ref,
                       "eps_measured_over_eps_ref": [st0.eps[q] / st0.eps_ref for q in range(st0.n_eps)],
                       "l2": "inputs larger than L2 (delta %d MB, phi %d MB)" % (8 * ng ** 3 >> 20, 8 * ng ** 3 >> 20),
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "gpu_launches": primary["launches"],
            "clocks": primary["clocks"],
            "roofline": roofline(primary, a.precision, fp64_tf),
            "alu_peaks_tflops": {"fp64": fp64_tf, "fp32": fp32_tf},
            "e2e": e2e_primary,
            "cpu_baseline": cb,
            "forms": forms}
    line["forms_summary"] = summarise(line, primary)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
