#!/usr/bin/env python
"""Benchmark of the finite-volume stage update (and the multigrid step) on GB300.

Headline: cell-updates/s per RK stage of the 2D Kelvin-Helmholtz workload
(2048^2 cells as 128x128 blocks of 16^2, HLLC + van Leer, SSPRK3, CFL 0.8,
periodic), FP32 batched path; the FP64 plain path is reported beside it.
A step = one SSPRK3 step = 3 stage launches (ghost gather, MUSCL, HLLC, flux
difference, SSPRK combination; the last one also does the CFL max-reduction
and the FP64 conserved totals), CUDA-graph launched.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the method runs all blocks on one GPU (no sharding, no collective);
N > 1 runs N independent replicas (weak scaling), value = sum over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage (KH 2048^2, FP32 batched)"
UNIT = "cell-stages/s"
NSIDE, BNX = 2048, 16
WORKLOAD = "2D Euler Kelvin-Helmholtz 2048^2, 128x128 blocks of 16^2, HLLC + van Leer, SSPRK3, CFL 0.8, periodic"


def kh_kwargs(nside=NSIDE, precision="fp32", stream=None):
    nb = nside // BNX
    return dict(ndim=2, block_nx=BNX, base=[nb, nb], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer",
                rk=3, bc="periodic", precision=precision, stream=stream)


def kh_state(lev, crd, nside=NSIDE, seed=2004):
    from paper_2004_03275_gb300 import inputs
    nb = nside // BNX
    x, gi = inputs.cell_centres(lev, crd, 2, BNX, [nb, nb, 1], [0, 0, 0], [1, 1, 1])
    return inputs.kelvin_helmholtz(x, gi, nside, seed=seed)


# Config 3 at a size the oracle finishes in seconds: base 2^3 blocks of 16^3, 3 levels (effective
# 128^3), 100 SSPRK3 steps with a regrid after every 10
BLAST128_BASE = [2, 2, 2]
BLAST128_KW = dict(ndim=3, block_nx=16, base=BLAST128_BASE, max_level=3, gamma=5.0 / 3.0, cfl=0.8, flux="hllc",
                   limiter="koren", rk=3, bc="periodic", refine_tol=0.2, coarsen_frac=0.5, var_mask=1 | 16)
BLAST128_STEPS, BLAST128_REGRID = 100, 10
# configuration 4's Gray-Scott parameters
GS_BATCH_KW = dict(Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5)


def blast_initial_refinement(g, base, max_level, seed=7):
    """Sample the blast on the tree, regrid, repeat (max_level passes): the same sequence for the
    oracle grid and the GPU solver."""
    from paper_2004_03275_gb300 import inputs
    for it in range(max_level):
        lev, crd = g.leaves()
        x, _ = inputs.cell_centres(lev, crd, 3, 16, base, [0, 0, 0], [1, 1, 1])
        g.set_prim(inputs.blast(x, seed=seed))
        if it < max_level - 1:
            g.regrid()


def fp32_accuracy_vs_oracle(amrvac, stream, ref):
    """Normalised L1(rho) of the float32 GPU path against the FP64 oracle states kept by the CPU
    baseline: the blast (effective 128^3, 100 steps with regrids; both runs regrid at the oracle's
    regrid times, both states projected to uniform 128^3) and KH 512^2 after 100 steps."""
    from paper_2004_03275_gb300 import analysis
    s = amrvac.AmrSolver(**BLAST128_KW, precision="fp32", stream=stream.cuda_stream)
    blast_initial_refinement(s, BLAST128_BASE, 3)
    nblk = len(ref["blast_marks"])
    for blk, t_mark in enumerate(ref["blast_marks"]):
        for _ in range(4):  # to the oracle's time (float32 dt may differ in the last digits)
            if s.t >= t_mark:
                break
            s.run(BLAST128_REGRID, t_end=t_mark)
            s.sync()
        if blk < nblk - 1:
            s.regrid()
    lev, crd = s.leaves()
    rho = analysis.project_uniform(lev, crd, s.read_state()[:, 0], 3, 16, BLAST128_BASE, 3)
    out = {"blast_128": {"l1_rho": analysis.l1_relative(rho, ref["blast_rho"]), "t": s.t,
                         "leaves": int(len(lev)),
                         "definition": "sum|rho32 - rho_oracle| / sum|rho_oracle| on uniform 128^3 after "
                                       f"{BLAST128_STEPS} steps, regrid every {BLAST128_REGRID}; both states "
                                       "projected (coarser leaves replicated)"}}
    s.close()
    kw = kh_kwargs(512, "fp32", stream.cuda_stream)
    s = amrvac.AmrSolver(**kw)
    lev, crd = s.leaves()
    s.set_prim(kh_state(lev, crd, 512))
    for _ in range(4):
        if s.t >= ref["kh512_t"]:
            break
        s.run(100, t_end=ref["kh512_t"])
        s.sync()
    out["kh_512"] = {"l1_rho": analysis.l1_relative(s.read_state()[:, 0], ref["kh512_rho"]), "t": s.t,
                     "definition": "sum|rho32 - rho_oracle| / sum|rho_oracle| after 100 steps (oracle's time)"}
    s.close()
    u0, v0 = ref["gs256_u0"]
    r = amrvac.RdSolver(2, [256], 2.5, precision="fp32", stream=stream.cuda_stream, **GS_BATCH_KW)
    r.set_state(u0.ravel(), v0.ravel())
    r.step(100)
    u32 = r.read_state()[0]
    r.close()
    out["gray_scott_256"] = {"l1_u": analysis.l1_relative(u32, ref["gs256_u"].ravel()),
                             "definition": "sum|u32 - u_oracle| / sum|u_oracle| after 100 IMEX steps (dt 0.5, "
                                           "multigrid rtol 1e-10) of the batch's 256^2 instance"}
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def bf16_peak():
    """Dense bf16 burst peak (TFLOP/s) from MEASURED_PEAKS.json, else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0))
    return 1900.0


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(dist, x, device):
    """Max of x over the ranks of the process group (identity without one); the timing of a
    replica run is the slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ws, ms_max):
    """Whole-job throughput of ws independent replicas: all ranks' units over the slowest time."""
    return ws * units_per_rank / (ms_max * 1e-3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def time_steps(torch, solver, stream, steps):
    """K graph-launched steps bracketed by synchronize, timed with CUDA events on the solver's stream."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    solver.run(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    solver.sync()
    return ev0.elapsed_time(ev1) / steps


# dram__bytes_read.sum + dram__bytes_write.sum per stage launch (mean of the three stages of a
# step) from the ncu capture of the stage kernel summarised in profiles/stage2d_march_kh2048.md;
# None when the kernel has changed since the counters were taken.
STAGE2D_F32_TRAFFIC = 144.8e6


def stage_roofline(solver, nsteps, nv, wbytes, ncells, hbm_gbs, ms_per_step, nstages=3, traffic=None):
    """Roofline of the stage kernel on a uniform grid, whose graph step holds only the nstages stage
    launches: the average launch duration is the graph-timed step over nstages (CUDA events on the
    launching stream around the timed region, so 3 x launch = step); algorithmic bytes per launch:
    stage 1 reads U^n and writes U^1 (2 nv w per cell), stages 2-3 read U^(s), U^n and write (3 nv w).
    Per-kernel event timings of a few extra steps (profile_step) are reported beside it."""
    bytes_step = (2 + 3 * (nstages - 1)) * nv * wbytes * ncells
    achieved = bytes_step / (ms_per_step * 1e-3) / 1e9
    ev = []
    for _ in range(nsteps):
        ev.append([ms for kind, ms in solver.profile_step() if kind == 0])
    ev = np.array(ev)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_gbs, "unit": "GB/s",
            "frac": round(achieved / hbm_gbs, 4), "traffic": traffic,
            "kernel": "stage2d_march_kernel<HLLC,VANLEER>", "launches_timed": "every stage launch of the timed steps",
            "avg_launch_us": round(ms_per_step * 1e3 / nstages, 2),
            "bytes_per_launch_avg": int(bytes_step / nstages), "frac_of_8TBs_nameplate": round(achieved / 8000, 4),
            "event_us_per_stage_kind": [round(float(v) * 1e3, 1) for v in np.median(ev, axis=0)]}


def bench_gray_scott(torch, amrvac, stream, steps=5):
    """Config 4: 16 Gray-Scott instances (256^2 .. 2048^2), IMEX steps, multigrid to 1e-10.
    Unit: cell-updates/s (both species of every instance per IMEX step)."""
    from paper_2004_03275_gb300 import inputs
    sizes = inputs.gray_scott_batch_sizes()
    us, vs = [], []
    for i, n in enumerate(sizes):
        u, v = inputs.gray_scott_patches(n, seed=4000 + i)
        us.append(u.ravel())
        vs.append(v.ravel())
    rd = amrvac.RdSolver(2, sizes, 2.5, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5, precision="fp32",
                         stream=stream.cuda_stream)
    rd.set_state(np.concatenate(us), np.concatenate(vs))
    rd.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cyc = rd.step(steps)
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / steps
    cells = sum(n * n for n in sizes)
    out = {"workload": "Gray-Scott IMEX, 16 instances 256^2..2048^2 (28.7M cells/species), dt 0.5, MG rtol 1e-10",
           "ms_per_step": el * 1e3, "cell_updates_per_s": 2 * cells / el, "steps": steps,
           "vcycles_per_solve_mean": float(np.mean(cyc)), "vcycles_max": int(np.max(cyc)),
           "timing": "host wall clock around rd_step (synchronous), stream synchronized"}
    rd.close()
    # accuracy of the FP32 path against the FP64 path (which matches the oracle, tests) after 100
    # steps of the whole batch (the oracle comparison of one instance is in the CPU-baseline leg)
    res = {}
    for prec in ("fp32", "fp64"):
        r = amrvac.RdSolver(2, sizes, 2.5, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5, precision=prec,
                            stream=stream.cuda_stream)
        r.set_state(np.concatenate(us), np.concatenate(vs))
        r.step(100)
        res[prec] = r.read_state()[0]
        r.close()
    du = np.abs(res["fp32"] - res["fp64"]).sum() / np.abs(res["fp64"]).sum()
    out["l1_u_fp32_vs_fp64_after_100_steps"] = float(du)
    return out


def _train_guess(torch, amrvac, LG, X, Y, ndim, loss, kappa, iters, batch):
    """One network trained with `loss`; the training-set loss of the zero output (the
    previous-step guess), of the initial network and of the trained one."""
    margin = LG.MARGIN[loss]
    zero = amrvac.CnnNet(ndim=ndim, seed=3)
    zero.set_params(np.zeros(zero.nparams, dtype=np.float32))
    zero.set_loss(loss, kappa)
    loss_zero = LG.dataset_loss(torch, zero, X, Y, margin=margin)
    zero.close()
    net = amrvac.CnnNet(ndim=ndim, seed=3)
    net.set_loss(loss, kappa)
    loss0 = LG.dataset_loss(torch, net, X, Y, margin=margin)
    _, train_s = LG.train(torch, net, X, Y, iters=iters, batch=batch, lr=1e-3, margin=margin)
    loss1 = LG.dataset_loss(torch, net, X, Y, margin=margin)
    return net, {"training_set_loss_zero_output_initial_trained": [loss_zero, loss0, loss1],
                 "train_s": round(train_s, 2)}


def bench_learned_guess(torch, amrvac, stream, eval_steps=6):
    """Config 5 (2D): learned multigrid guesses trained on crops of 2048^2 runs (training seeds 0, 1),
    evaluated at 2048^2 on seed 10000 against the previous-step guess.  Two networks:
    * residual inputs (the normalised residual of the previous-step guess) trained on the
      operator-weighted loss (the guess's own residual);
    * (u*_prev, v*_prev) inputs trained on the masked MSE of the increment."""
    from paper_2004_03275_gb300 import learned_guess as LG
    n, L = 2048, 2.5
    kappa = LG.operator_kappa(n, L, ndim=2)
    c0, t0s, _, r0 = LG.evaluate(torch, [n], [10000], L, steps=eval_steps, warm=40)
    out = {"workload": "Gray-Scott IMEX 2048^2 (seed 10000, after 40 warm-up steps), MG rtol 1e-10",
           "training_data": "crops 64^2 after each of 24 steps of two 2048^2 runs (seeds 0, 1; 40 warm-up steps), "
                            "48 crops per step (1152 pairs); the 20000-pair entry: 100 steps, 200 crops per step",
           "vcycles_per_solve_previous_step_guess": float(np.mean(c0)),
           "initial_rel_residual_median_previous_step": float(np.median(r0)),
           "ms_per_step_previous_step_guess": t0s * 1e3, "operator_kappa": [round(k, 5) for k in kappa]}
    # (inputs, loss, Adam steps, crops per step, steps): the two networks on 1152 crops, and the
    # residual network on the configuration's 20k training pairs (100 steps x 200 crops of the two runs)
    for inp, loss, iters, cps, nst in (("residual", "operator", 5000, 48, 24), ("prev", "mse", 1500, 48, 24),
                                       ("residual", "operator", 5000, 200, 100)):
        t0 = time.perf_counter()
        X, Y, scale = LG.generate(torch, [n, n], [0, 1], L, steps=nst, crops_per_step=cps, crop=64, warm=40,
                                  inputs=inp)
        gen_s = time.perf_counter() - t0
        net, info = _train_guess(torch, amrvac, LG, X, Y, 2, loss, kappa, iters=iters, batch=64)
        c1, t1s, _, r1 = LG.evaluate(torch, [n], [10000], L, steps=eval_steps, warm=40, net=net, scale=scale,
                                     inputs=inp)
        info.update({"data_s": round(gen_s, 2), "training_pairs": int(X.shape[0]), "adam_steps": iters, "batch": 64,
                     "lr": 1e-3,
                     "vcycles_per_solve": float(np.mean(c1)), "vcycles_per_solve_each": [int(x) for x in c1.ravel()],
                     "initial_rel_residual_median": float(np.median(r1)), "ms_per_step": t1s * 1e3,
                     "cnn_launches": net.kernel_launches()})
        out[f"learned_{inp}_inputs_{loss}_loss_{int(X.shape[0])}_pairs"] = info
        net.close()
        del X, Y
    return out


def bench_learned_guess_3d(torch, amrvac, stream, eval_steps=6):
    """Config 5 (3D): the learned guess ((u*_prev, v*_prev) inputs, masked MSE) trained on crops of
    256^3 runs (training seeds 0, 1), evaluated at 256^3 on seed 10000 against the previous-step guess."""
    from paper_2004_03275_gb300 import learned_guess as LG
    N, L = 256, 2.5
    t0 = time.perf_counter()
    X, Y, scale = LG.generate(torch, [N, N], [0, 1], L, steps=16, crops_per_step=12, crop=32, warm=20, ndim=3)
    gen_s = time.perf_counter() - t0
    c0, t0s, _, r0 = LG.evaluate(torch, [N], [10000], L, steps=eval_steps, warm=20, ndim=3)
    net, info = _train_guess(torch, amrvac, LG, X, Y, 3, "mse", None, iters=600, batch=4)
    c1, t1s, _, r1 = LG.evaluate(torch, [N], [10000], L, steps=eval_steps, warm=20, net=net, scale=scale, ndim=3)
    net.close()
    info.update({"vcycles_per_solve": float(np.mean(c1)), "initial_rel_residual_median": float(np.median(r1)),
                 "ms_per_step": t1s * 1e3})
    return {"workload": "Gray-Scott IMEX 256^3 on [0,2.5]^3 (seed 10000, after 20 warm-up steps), MG rtol 1e-10",
            "training": f"{X.shape[0]} crops 32^3 after each of 16 steps of two 256^3 runs (seeds 0, 1), "
                        f"{gen_s:.1f}s; 600 Adam steps, batch 4, lr 1e-3",
            "vcycles_per_solve_previous_step_guess": float(np.mean(c0)),
            "initial_rel_residual_median_previous_step": float(np.median(r0)),
            "ms_per_step_previous_step_guess": t0s * 1e3, "learned_prev_inputs_mse_loss": info}


# Algorithmic bytes per level-0 unknown per V-cycle of the float32 multigrid (nu1 = nu2 = 2, 2D):
#   level 0: 4 sweeps x (read x, b; write x: 12 B) = 48; residual + restriction (read x0, b0; write 1/4
#   of b1, x1) = 10; prolongation (read 1/4 of x1, read + write x0) = 9; float64 correction and defect
#   update (read x0, X, R; write X, R, b0) = 40; correction zeroed (write x0) = 4  -> 111 B;
#   coarser levels: (48 + 10 + 9) B x (1/4 + 1/16 + ...) = 22 B  -> 133 B.
MG_BYTES_PER_UNKNOWN_VCYCLE = 133.0


def bench_mg_vcycle(torch, amrvac, stream, hbm_gbs):
    """Time of one V-cycle of the batched float32 multigrid over the configuration-4 instance sizes
    (16 grids 256^2..2048^2, 28.7M unknowns, lambda = 2/(dt Du) of Gray-Scott's u): two solves from a
    zero guess to rtol 1e-3 and 1e-12 (best of 5 each), differenced, so the per-solve setup cancels."""
    from paper_2004_03275_gb300 import inputs
    sizes = inputs.gray_scott_batch_sizes()
    n = sum(k * k for k in sizes)
    lam = 2.0 / (0.5 * 2e-5)
    b = torch.from_numpy(np.random.default_rng(7).normal(size=n)).cuda()
    res = {}
    for rtol in (1e-3, 1e-12):
        s = amrvac.MgSolver(2, sizes, lam, 2.5, rtol=rtol, precision="fp32", stream=stream.cuda_stream)
        x = torch.zeros_like(b)
        s.solve(b, x)
        best = None
        for _ in range(5):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cyc, _ = s.solve(b, x)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            best = el if best is None else min(best, el)
        res[rtol] = (best, int(np.max(cyc)))
        if rtol == 1e-12:  # one V-cycle kernel by kernel (CUDA events between launches), 5 times
            with torch.cuda.nvtx.range("mg_profile_vcycle"):
                prof = [s.profile_vcycle() for _ in range(6)][1:]
        s.close()
    kinds = {}
    for p in prof:
        for k, us in p:
            kinds.setdefault(k, [0, 0.0])
            kinds[k][0] += 1
            kinds[k][1] += us / len(prof)
    tot = sum(v[1] for v in kinds.values())
    # the first launch is depth 0's first pre-sweep over every instance: 12 B per unknown
    sweep0 = float(np.mean([p[0][1] for p in prof]))
    (t_lo, c_lo), (t_hi, c_hi) = res[1e-3], res[1e-12]
    tv = (t_hi - t_lo) / max(1, c_hi - c_lo)
    gbs = MG_BYTES_PER_UNKNOWN_VCYCLE * n / tv / 1e9
    return {"workload": "batched Helmholtz multigrid, 16 periodic grids 256^2..2048^2 (28.7M unknowns), "
                        "float32 V-cycles on the float64 defect, nu1 = nu2 = 2",
            "ms_per_vcycle": tv * 1e3, "unknown_vcycles_per_s": n / tv, "cycles_rtol_1e-3_1e-12": [c_lo, c_hi],
            "roofline": {"bound": "hbm", "bytes_per_unknown": MG_BYTES_PER_UNKNOWN_VCYCLE,
                         "achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s", "frac": round(gbs / hbm_gbs, 4)},
            "timing": "host wall clock around synchronous solves (includes the per-cycle residual check and "
                      "host poll), best of 5, difference of two tolerances",
            "kernels_of_one_vcycle": {"us_by_kind": {k: round(v[1], 1) for k, v in kinds.items()},
                                      "launches_by_kind": {k: v[0] // len(prof) for k, v in kinds.items()},
                                      "sum_us": round(tot, 1),
                                      "depth0_sweep_us": round(sweep0, 1),
                                      "sequence_us": [[k, round(float(np.mean([p[i][1] for p in prof])), 1)]
                                                      for i, (k, _) in enumerate(prof[0])],
                                      "depth0_sweep_gbs": round(12.0 * n / (sweep0 * 1e-6) / 1e9, 1),
                                      "timing": "mg_profile_vcycle: kernels launched one by one with CUDA events "
                                                "between them (not graph-replayed), mean of 5 cycles"}}


def bench_schnakenberg(torch, amrvac, stream):
    """Sec. 2.5.2's Schnakenberg study on the GPU: Eq. (schnakenberg) with D_u = 0.05, D_v = 1,
    kappa = 100, a = 0.1305, b = 0.7695 on [0, 1]^d with zero-flux boundaries.
    (1) Time per step of the explicit, IMEX and split schemes at 256^2 (the paper: 1.1, 7.7 and
    7.2 ms on 4 CPU cores, multigrid to 1e-7 of the right-hand side) and at 128^3: explicit at
    dt = 3e-6 (2D) / 1e-5 (3D), below h^2 / (2 ndim D_v); IMEX and split at dt = 1e-3.
    (2) The paper's convergence study: 256^2 at t = 2 against an explicit run with dt = 3e-6
    (666,667 steps), multigrid to 1e-10; IMEX at dt = 4e-3 .. 5e-4, split at dt = 1e-3 .. 1.25e-4
    (its forward-Euler reaction step is unstable above dt ~ 1.1e-3: the reaction Jacobian at the
    homogeneous steady state has eigenvalues -3.55 +- 80.4i)."""
    from paper_2004_03275_gb300 import inputs
    P = inputs.SCHNAKENBERG
    kw = dict(Du=P["Du"], Dv=P["Dv"], kappa=P["kappa"], a=P["a"], b=P["b"], model="schnakenberg", bc="neumann",
              precision="fp32", stream=stream.cuda_stream)

    def solver(ndim, n, scheme, dt, rtol):
        u0, v0 = inputs.schnakenberg_initial(n, ndim)
        s = amrvac.RdSolver(ndim, [n], 1.0, dt=dt, scheme=scheme, rtol=rtol, **kw)
        s.set_state(u0.ravel(), v0.ravel())
        return s

    timing = {}
    for ndim, n in ((2, 256), (3, 128)):
        for scheme, dt, steps in (("explicit", 3e-6 if ndim == 2 else 1e-5, 4000), ("imex", 1e-3, 100),
                                  ("split", 1e-3, 100)):
            s = solver(ndim, n, scheme, dt, 1e-7)
            s.step(steps // 10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cyc = s.step(steps)
            el = (time.perf_counter() - t0) / steps
            timing[f"{scheme}_{n}^{ndim}"] = {"dt": dt, "ms_per_step": round(el * 1e3, 5),
                                              "vcycles_per_solve": round(float(np.mean(cyc)), 2)}
            s.close()
    T = 2.0
    s = solver(2, 256, "explicit", 3e-6, 1e-10)
    nref = int(round(T / 3e-6))
    t0 = time.perf_counter()
    s.step(nref)
    t_ref = time.perf_counter() - t0
    ur, vr = s.read_state()
    s.close()
    conv = {}
    for scheme, dts in (("imex", (4e-3, 2e-3, 1e-3, 5e-4)), ("split", (1e-3, 5e-4, 2.5e-4, 1.25e-4))):
        errs = []
        for dt in dts:
            s = solver(2, 256, scheme, dt, 1e-10)
            s.step(int(round(T / dt)))
            u, v = s.read_state()
            errs.append(float(np.sqrt(np.mean((u - ur) ** 2 + (v - vr) ** 2))))
            s.close()
        e = np.array(errs)
        conv[scheme] = {"dt": list(dts), "l2_error": errs,
                        "orders": [round(float(x), 3) for x in np.log2(e[:-1] / e[1:])]}
    return {"workload": "Schnakenberg (Sec. 2.5.2), Neumann, L = 1, 256^2 and 128^3, float32 multigrid on the "
                        "float64 defect, state float64",
            "per_step": timing,
            "paper_per_step_ms_256^2_4_cpu_cores": {"explicit": 1.1, "imex": 7.7, "split": 7.2},
            "convergence_t2_256^2": conv, "reference_explicit_steps": nref, "reference_seconds": round(t_ref, 2),
            "timing": "host wall clock around synchronous rd_step calls"}


def bench_gray_scott_tree(torch, amrvac, stream, steps=40, regrid_every=10):
    """Sec. 2.5.2's Gray-Scott run on an adaptive three-level block quadtree: F = 0.046,
    k = 0.063, D_u = 2e-5, D_v = 1e-5, L = 2, 8^2 blocks, base 128^2, finest 512^2, dt = 0.5, two
    Gaussian perturbations; IMEX steps with the float64 tree multigrid (rtol 1e-10) and a regrid
    (Lohner estimator of u, refine above 0.01, coarsen below 0.005) every 10 steps."""
    from paper_2004_03275_gb300 import inputs
    p = inputs.GRAY_SCOTT_PAPER
    nb, B = 16, 8
    lev, crd = inputs.gray_scott_tree(nb=nb, L=p["L"])
    X, Y = inputs.leaf_cell_centres(lev, crd, nb, B, p["L"])
    u, v = inputs.gray_scott_gaussians(X, Y)
    s = amrvac.TreeRdSolver(lev, crd, nb, B, p["L"], Du=p["Du"], Dv=p["Dv"], F=p["F"], k=p["k"], dt=p["dt"],
                            stream=stream.cuda_stream)
    s.set_state(u.ravel(), v.ravel())
    s.step(2)
    n0 = s.kernel_launches()
    per_level, t_step, t_regrid, cyc = [], 0.0, 0.0, []
    torch.cuda.synchronize()
    for k in range(steps // regrid_every):
        t0 = time.perf_counter()
        cyc.append(s.step(regrid_every))
        t1 = time.perf_counter()
        s.regrid(refine_tol=0.01, coarsen_frac=0.5, max_level=3)
        t2 = time.perf_counter()
        t_step += t1 - t0
        t_regrid += t2 - t1
        per_level.append([int(c) for c in np.bincount(s.leaves()[0], minlength=4)[1:]])
    out = {"workload": "Gray-Scott IMEX on an adaptive 3-level quadtree (8^2 blocks, 128^2..512^2), float64 tree "
                       "multigrid, regrid every 10 steps",
           "initial_leaves_per_level": [int(c) for c in np.bincount(lev)[1:]], "leaves_per_level_after_each_regrid": per_level,
           "ms_per_step": round(t_step / steps * 1e3, 3), "ms_per_regrid": round(t_regrid / (steps // regrid_every) * 1e3, 2),
           "vcycles_per_solve": round(float(np.mean(np.concatenate(cyc))), 2),
           "kernels_per_step_incl_regrids": round((s.kernel_launches() - n0) / steps, 1), "steps": steps,
           "timing": "host wall clock around synchronous rdt_step / rdt_regrid calls (each solve one graph with "
                     "device-side loops)"}
    s.close()
    return out


# 2 x 9 x (5*16 + 16*16 + 16*16 + 16*2) multiply-adds x 2 per pixel for the 4 layers
CNN_FLOP_PER_PIXEL_2D = 11232.0
# HBM bytes per pixel of the layer-by-layer inference: layer 1 reads the float32 5-channel input
# (20 B) and writes 16 bf16 channels (32 B); layers 2-3 read and write 32 B; layer 4 reads 32 B
# and writes 2 float32 channels (8 B).  51 FLOP/B overall, below GB300's ~285 FLOP/B ridge
# (measured bf16 peak / measured HBM bandwidth), so the attainable roofline is the HBM one.
CNN_BYTES_PER_PIXEL_2D = 52.0 + 64.0 + 64.0 + 40.0
# the fused inference reads the five float32 input channels and writes the two float32 outputs
CNN_FUSED_BYTES_PER_PIXEL_2D = 5 * 4.0 + 2 * 4.0


def bench_cnn_forward(torch, amrvac, stream, peak_tflops, hbm_gbs):
    """Inference of the learned-guess network on one 2048^2 grid (5 input channels), CUDA events:
    the fused single-pass kernel (cnn_infer; the inference the solver's guess runs) and the
    layer-by-layer network (cnn_forward, exact GELU; the training forward pass)."""
    net = amrvac.CnnNet(ndim=2, seed=3, stream=stream.cuda_stream)
    x = torch.from_numpy(np.random.default_rng(3).uniform(size=(1, 5, 2048, 2048)).astype(np.float32)).cuda()
    out = torch.empty((1, 2, 2048, 2048), dtype=torch.float32, device="cuda")
    px = 2048 * 2048

    def timed(fn, reps=20):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn(x, out)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                fn(x, out)
            ev1.record(stream)
            torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    ms_fused = timed(net.infer)
    ms_layers = timed(net.forward)
    net.close()
    tf = CNN_FLOP_PER_PIXEL_2D * px / (ms_fused * 1e-3) / 1e12
    gbs = CNN_FUSED_BYTES_PER_PIXEL_2D * px / (ms_fused * 1e-3) / 1e9
    return {"workload": "learned-guess CNN inference, 2048^2, 5->16->16->16->2 channels, 3x3, bf16 mma.sync",
            "ms_per_inference": ms_fused, "kernel": "cnn_fused2d_kernel (all four layers in one pass)",
            "ms_per_inference_layer_by_layer": ms_layers,
            "tensor": {"achieved_tflops": round(tf, 1), "peak_tflops": peak_tflops, "frac": round(tf / peak_tflops, 4),
                       "flop_per_pixel": CNN_FLOP_PER_PIXEL_2D},
            "hbm": {"achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s", "frac": round(gbs / hbm_gbs, 4),
                    "bytes_per_pixel": CNN_FUSED_BYTES_PER_PIXEL_2D}}


def bench_blast(torch, amrvac, stream, hbm_gbs, steps=20, regrid_every=10):
    """Config 3: 3D blast, 4^3 base blocks of 16^3, 4 levels (effective 512^3), HLLC + Koren, SSPRK3,
    FP32 state, regrid every 10 steps.  cell-updates/s per RK stage excluding regrid time."""
    from paper_2004_03275_gb300 import inputs
    kw = dict(ndim=3, block_nx=16, base=[4, 4, 4], max_level=4, gamma=5.0 / 3.0, cfl=0.8, flux="hllc",
              limiter="koren", rk=3, bc="periodic", refine_tol=0.2, coarsen_frac=0.5, var_mask=1 | 16,
              precision="fp32", max_blocks=20000, stream=stream.cuda_stream)
    s = amrvac.AmrSolver(**kw)
    blast_initial_refinement(s, [4, 4, 4], 4)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, cells_steps, t_regrid, levels = 0.0, 0, 0.0, []
    done = 0
    while done < steps:
        k = min(regrid_every, steps - done)
        lev, _ = s.leaves()
        levels.append(np.bincount(lev, minlength=5)[1:].tolist())
        torch.cuda.synchronize()
        ev0.record(stream)
        s.run(k)
        ev1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        step_ms += ev0.elapsed_time(ev1)
        cells_steps += len(lev) * 4096 * k
        done += k
        t0 = time.perf_counter()
        s.regrid()
        t_regrid += time.perf_counter() - t0
    rate = 3 * cells_steps / (step_ms * 1e-3)
    # algorithmic bytes per cell-stage, SSPRK3 mean: (2 + 3 + 3) / 3 stages x 5 variables x 4 bytes
    bps = 8.0 / 3.0 * 5 * 4
    out = {"workload": "3D blast, base 4^3 x 16^3, max_level 4 (eff. 512^3), HLLC+Koren, SSPRK3, FP32",
           "steps": steps, "cell_stage_updates_per_s": rate,
           "ms_per_step_mean": step_ms / steps, "regrid_ms_mean": t_regrid * 1e3 / max(1, steps // regrid_every),
           "blocks_per_level_at_each_regrid": levels,
           "roofline": {"bound": "hbm", "bytes_per_cell_stage": round(bps, 2), "achieved": round(rate * bps / 1e9, 1),
                        "peak": hbm_gbs, "unit": "GB/s", "frac": round(rate * bps / 1e9 / hbm_gbs, 4),
                        "scope": "whole step: stage passes, level-jump ghost fill, reflux, reductions; regrid excluded"}}
    s.close()
    # accuracy of the FP32 path: both precisions on the same tree (built by the FP64 solver) and
    # initial state, 10 steps without regrid; the FP64 GPU path matches the oracle (tests)
    k64 = dict(kw, precision="fp64")
    s64 = amrvac.AmrSolver(**k64)
    for it in range(4):
        lev, crd = s64.leaves()
        x, _ = inputs.cell_centres(lev, crd, 3, 16, [4, 4, 4], [0, 0, 0], [1, 1, 1])
        V = inputs.blast(x, seed=7)
        s64.set_prim(V)
        if it < 3:
            s64.regrid()
    s32 = amrvac.AmrSolver(**kw)
    s32.set_leaves(lev, crd)
    s32.set_prim(V)
    s64.run(10)
    s64.sync()
    for _ in range(4):  # to the FP64 path's time (float32 dt may differ in the last digits)
        if s32.t >= s64.t:
            break
        s32.run(10, t_end=s64.t)
        s32.sync()
    r64, r32 = s64.read_state()[:, 0], s32.read_state()[:, 0]
    out["l1_rho_fp32_vs_fp64_10_steps"] = float(np.abs(r32 - r64).sum() / np.abs(r64).sum())
    s64.close()
    s32.close()
    return out


def _oracle_kh_rate(O, side, budget_s):
    """cell-stages/s of the oracle on KH side^2 (SSPRK3 steps until budget_s has passed)."""
    kw = kh_kwargs(side)
    kw.pop("precision")
    kw.pop("stream")
    g = O.Grid(**kw)
    lev, crd = g.leaves()
    g.set_prim(kh_state(lev, crd, side))
    t0 = time.perf_counter()
    n = 0
    while True:
        g.step()
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return side * side * 3 * n / el, n, el


def oracle_cpu_baseline(budget_s=8.0):
    """The FP64 oracle as it stands on the host cores: KH on one thread and on all cores (its
    OpenMP loops over blocks give the one-thread result bit for bit), plus bounded samples of
    the batched multigrid V-cycle and of the 3D blast tree on all cores.  Returns the report and
    the oracle states (blast and KH 512^2) that the float32 accuracy figures are taken against."""
    import oracle as O
    nproc = os.cpu_count() or 1
    O.set_threads(1)
    v1, n1, el1 = _oracle_kh_rate(O, 512, budget_s)
    O.set_threads(nproc)
    vn, nn, eln = _oracle_kh_rate(O, 1024, budget_s)
    out = {"value": vn, "unit": UNIT, "cores": nproc, "nproc": nproc, "kind": "oracle",
           "sample": f"KH 1024^2 (4096 blocks of 16^2), {nn} SSPRK3 steps, FP64, {nproc} threads, {eln:.1f} s",
           "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                             "sample": f"KH 512^2, {n1} SSPRK3 steps, FP64, 1 thread, {el1:.1f} s"}}
    # multigrid: V-cycles of the oracle on one 1024^2 periodic grid (lambda of the Gray-Scott u
    # species at 2048^2), unknown-V-cycles/s, one thread and all cores
    n = 1024
    r = np.random.default_rng(7).standard_normal((n, n))
    lam = 2.0 / (0.5 * 2e-5)
    mg = {}
    for th in (1, nproc):
        O.set_threads(th)
        t0 = time.perf_counter()
        k = 0
        while k < 2 or time.perf_counter() - t0 < budget_s / 2:
            O.mg_vcycle(r, 2.5 * n / 2048, lam)
            k += 1
        el = time.perf_counter() - t0
        mg[f"threads_{th}"] = {"value": n * n * k / el, "unit": "unknown-V-cycles/s", "vcycles": k,
                               "seconds": round(el, 2)}
    out["mg_vcycle"] = dict(mg, sample="FP64 V-cycles (2 + 2 red-black sweeps) on one periodic 1024^2 grid")
    # blast: base 2^3 blocks of 16^3, 3 levels (effective 128^3), initial refinement, then 100
    # SSPRK3 steps with a regrid after every 10 (regrids not timed), all cores.  The final state
    # and the regrid times are kept for the float32 GPU run of the same configuration.
    from paper_2004_03275_gb300 import analysis
    g = O.Grid(**BLAST128_KW)
    blast_initial_refinement(g, BLAST128_BASE, 3)
    el, cell_stages, marks, leaves = 0.0, 0, [], []
    for blk in range(BLAST128_STEPS // BLAST128_REGRID):
        leaves.append(g.nleaves)
        t0 = time.perf_counter()
        k = g.run(BLAST128_REGRID)
        el += time.perf_counter() - t0
        cell_stages += g.nleaves * 16 ** 3 * 3 * k
        marks.append(g.t)
        if blk < BLAST128_STEPS // BLAST128_REGRID - 1:
            g.regrid()
    lev, crd = g.leaves()
    rho = analysis.project_uniform(lev, crd, g.get_cons()[:, 0], 3, 16, BLAST128_BASE, 3)
    out["blast3d"] = {"value": cell_stages / el, "unit": UNIT, "cores": nproc, "leaves_per_block_of_10_steps": leaves,
                      "sample": f"blast, 2^3 base blocks of 16^3, 3 levels (effective 128^3), {BLAST128_STEPS} SSPRK3 "
                                f"steps with a regrid every {BLAST128_REGRID} (not timed), {nproc} threads, "
                                f"{el:.1f} s", "t_end": g.t}
    # Gray-Scott, the batch's 256^2 instance (seed 4000), 100 IMEX steps: the reference of the
    # float32 multigrid path's accuracy figure
    from paper_2004_03275_gb300 import inputs as _inp
    u0, v0 = _inp.gray_scott_patches(256, seed=4000)
    ug, vg = u0.copy(), v0.copy()
    for _ in range(100):
        ug, vg, _c = O.rd_step(ug, vg, 2.5, **GS_BATCH_KW)
    # KH 512^2, 100 steps, all cores: the reference state of the float32 accuracy figure
    kw = kh_kwargs(512)
    kw.pop("precision")
    kw.pop("stream")
    gk = O.Grid(**kw)
    lev, crd = gk.leaves()
    gk.set_prim(kh_state(lev, crd, 512))
    gk.run(100)
    return out, {"blast_marks": marks, "blast_rho": rho, "kh512_t": gk.t, "kh512_rho": gk.get_cons()[:, 0].copy(),
                 "kh512_leaves": (lev, crd), "gs256_u0": (u0, v0), "gs256_u": ug}


def run_reference(args, ws, rank):
    """--impl reference: the oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return 0
    import oracle as O
    nproc = os.cpu_count() or 1
    O.set_threads(nproc)
    total = args.steps + args.warmup
    budget = 150.0 / max(total, 1)  # seconds per step so that the run stays within a few minutes
    side = 32
    for s in (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048):
        if s * s * 3 * 1.0e-6 / nproc <= budget:  # ~1 us per cell-stage on one core
            side = s
    kw = kh_kwargs(side)
    kw.pop("precision")
    kw.pop("stream")
    g = O.Grid(**kw)
    lev, crd = g.leaves()
    g.set_prim(kh_state(lev, crd, side))
    for _ in range(args.warmup):
        g.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.step()
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = side * side * 3 / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_side": side, "parallelism": f"cpu oracle, {nproc} threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
                             "sample": f"KH {side}^2 per step (bounded sample of the 2048^2 workload)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-extra", action="store_true", help="skip the Gray-Scott and blast configurations")
    ap.add_argument("--extras", default="all",
                    help="comma list of extra workloads: gray_scott_batch, mg_vcycle, blast3d, learned_guess_2d, "
                         "learned_guess_3d, cnn_forward_2048 (default all; 'none' for none)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2004_03275_gb300 import amrvac

    amrvac.load()  # fails loudly if the CUDA library is missing
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(dist, x, "cuda")

    # a real (non-legacy) stream shared by the library and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    hbm, peak_src = peaks()
    ncells = NSIDE * NSIDE

    # ---------------------------------------------------------------- FP32 headline
    s32 = amrvac.AmrSolver(**kh_kwargs(precision="fp32", stream=stream.cuda_stream))
    lev, crd = s32.leaves()
    V = kh_state(lev, crd)
    s32.set_prim(V)
    s32.run(args.warmup)
    s32.sync()
    clk = Clocks(local)
    if rank == 0:
        clk.start()
    barrier()
    l0 = s32.kernel_launches()
    with torch.cuda.nvtx.range("kh_timed_steps"):  # a profiler can select the timed launches by it
        ms32 = time_steps(torch, s32, stream, args.steps)
    launches = s32.kernel_launches() - l0
    barrier()
    clocks = clk.stop() if rank == 0 else None
    ms32 = max_over_ranks(ms32)
    value = replica_value(ncells * 3, ws, ms32)
    roof = stage_roofline(s32, 5, 4, 4, ncells, hbm, ms32, traffic=STAGE2D_F32_TRAFFIC)
    roof["peak_source"] = peak_src
    pick, pick_us = s32.march_tuning()
    roof["tuned_launch"] = {kind: {"warps_per_cta": nw, "persistent": bool(p), "us": round(u, 2)}
                            for kind, (nw, p), u in zip(("first", "middle", "last"), pick, pick_us)}

    # ---------------------------------------------------------------- FP64 plain
    fp64 = None
    if not args.skip_fp64:
        s64 = amrvac.AmrSolver(**kh_kwargs(precision="fp64", stream=stream.cuda_stream))
        s64.set_prim(V)
        s64.run(3)
        s64.sync()
        k64 = max(3, min(200, args.steps // 20))
        barrier()
        ms64 = max_over_ranks(time_steps(torch, s64, stream, k64))
        r64 = stage_roofline(s64, 2, 4, 8, ncells, hbm, ms64)
        fp64 = {"value": ws * ncells * 3 / (ms64 * 1e-3), "ms_per_step": ms64, "steps": k64,
                "stage_achieved_gbs": r64["achieved"], "stage_frac_hbm": r64["frac"],
                "fp32_over_fp64": (ms64 / ms32)}
        # accuracy of the FP32 path: both paths from the initial state to the time the FP64 path
        # reaches in 100 steps (the configuration's run length); the FP64 GPU path matches the
        # FP64 oracle to 1e-12 per cell (tests), so it stands in for the oracle at this size
        if rank == 0:
            s64.set_prim(V)
            s64.set_time(0.0)
            s64.run(100)
            s64.sync()
            t100 = s64.t
            r64s = s64.read_state()[:, 0]
            a32 = amrvac.AmrSolver(**kh_kwargs(precision="fp32", stream=stream.cuda_stream))
            a32.set_prim(V)
            for _ in range(4):
                if a32.t >= t100:
                    break
                a32.run(100, t_end=t100)
                a32.sync()
            r32s = a32.read_state()[:, 0]
            fp64["l1_rho_fp32_vs_fp64"] = float(np.abs(r32s - r64s).sum() / np.abs(r64s).sum())
            fp64["l1_at"] = {"t": t100, "fp64_steps": 100, "t_fp32": a32.t}
            a32.close()
        s64.close()

    # ---------------------------------------------------------------- end to end
    e2e = None
    if not args.skip_e2e:
        U = s32.read_state()
        nbytes = U.size * 8
        hin = torch.from_numpy(U.reshape(-1).copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        k = max(3, min(20, args.steps // 100))
        s32.set_state(hin, primitive=False)
        s32.run(1)
        s32.read_state(hout.view(U.shape))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            s32.set_state(hin, primitive=False)  # H2D of the step's input (pinned, float64)
            s32.run(1)
            s32.read_state(hout.view(U.shape))   # D2H of the step's result (float64)
        torch.cuda.synchronize()
        el = max_over_ranks((time.perf_counter() - t0) / k)
        e2e = {"value": ws * ncells * 3 / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": el * 1e3,
               "path": "amr_set_state(host) + amr_run(1) + amr_read_state(host), float64 conserved state"}

    totals = s32.totals().tolist()
    s32.close()

    extra = {}
    if not args.skip_extra and rank == 0:
        names = ["gray_scott_batch", "mg_vcycle", "blast3d", "learned_guess_2d", "learned_guess_3d",
                 "cnn_forward_2048", "schnakenberg", "gray_scott_tree"]
        want = names if args.extras == "all" else [e for e in args.extras.split(",") if e in names]
        runs = {"gray_scott_batch": lambda: bench_gray_scott(torch, amrvac, stream),
                "mg_vcycle": lambda: bench_mg_vcycle(torch, amrvac, stream, hbm),
                "blast3d": lambda: bench_blast(torch, amrvac, stream, hbm),
                "learned_guess_2d": lambda: bench_learned_guess(torch, amrvac, stream),
                "learned_guess_3d": lambda: bench_learned_guess_3d(torch, amrvac, stream),
                "cnn_forward_2048": lambda: bench_cnn_forward(torch, amrvac, stream, bf16_peak(), hbm),
                "schnakenberg": lambda: bench_schnakenberg(torch, amrvac, stream),
                "gray_scott_tree": lambda: bench_gray_scott_tree(torch, amrvac, stream)}
        for name in want:
            # an extra workload that fails is reported as such; the headline line still prints;
            # each runs inside an NVTX range of its name (a profiler can select one by it)
            try:
                with torch.cuda.nvtx.range(name):
                    extra[name] = runs[name]()
            except Exception as e:  # noqa: BLE001
                extra[name] = {"error": f"{type(e).__name__}: {e}"[:500]}

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu, ref = oracle_cpu_baseline()
        try:
            cpu["fp32_accuracy_vs_oracle"] = fp32_accuracy_vs_oracle(amrvac, stream, ref)
        except Exception as e:  # noqa: BLE001
            cpu["fp32_accuracy_vs_oracle"] = {"error": f"{type(e).__name__}: {e}"[:500]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": ncells, "stages_per_step": 3, "seed": 2004,
                       "l2": "no flush: per-stage working set 201 MB (3 float32 state arrays) > 129 MB L2",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU, all blocks resident"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "fp64_plain": fp64, "totals_fp64": totals,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
