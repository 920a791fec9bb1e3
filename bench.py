"""Benchmark: HWENO-GR SSP-RK3 time steps on the viscous shock tube (1024 x 512).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hweno|reference]

A step is one SSP-RK3 time step (three evaluations of the spatial operator, three
stage updates, the time-step rule and the admissibility check) of the 1024 x 512
viscous shock-tube workload (no-slip walls, symmetry plane, Re 1000, Pr 0.73).
The metric is Gcell-RK-stage/s = cells x stages / seconds, summed over ranks.

  value     device-resident state, CUDA-event time of K steps (FP64 path)
  e2e       the same steps through the C ABI with host buffers: each step loads
            the state from pinned host memory and reads the new state back
  mixed     the FP32-reconstruction path on the same steps, with its L1 error
            against the FP64 path after the K steps and its roofline
  dr        the paper's comparison scheme HWENO-DR (differentiated candidates for
            the viscous gradients) on the same workload and steps, FP64
  roofline  the dominant kernel's algorithmic FP64 flops per launch (the oracle's
            operation count per interior cell) / its mean event-timed duration,
            against the FP64 FMA peak measured live; the whole step on the same basis
  adjoint   the gradient of a final-time misfit through 200 steps of the
            512^2 Taylor-Green flow, checkpoints every 20; backward / forward time and
            central differences on 16 seeded directions
  ensemble  64 Taylor-Green cases (sides 128-1024) in batched mixed steps,
            with the worst case's error against FP64
  colliding_streams  the 2048^2 near-vacuum colliding streams, FP64 and
            mixed
  mms       Example 5.2's manufactured-source study at 40^2 and 80^2, GR and DR:
            density errors against the exact solution and their orders
  cpu_baseline  the FP64 CPU oracle on the host cores, one SSP-RK3 step of the
            same workload (rank 0, N = 1 only)

--impl reference times the CPU oracle (the only other implementation of the
method) on full-size steps of the same workload, as many as fit a bounded time.

Multi-GPU: independent replicas, one per rank (torchrun), no collective in the
data path; the barrier and max-over-ranks timing use torch.distributed.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-RK-stage/s"
WORKLOAD = "viscous shock tube 1024x512, no-slip walls + symmetry, Re 1000, Pr 0.73, SSP-RK3 under the CFL/viscous step rule"

# Algorithmic floating-point work per interior cell and RK stage, by phase of the
# spatial operator: the distinct state-dependent additions, multiplications, divisions
# and square roots of the FP64 oracle's own algebra (each candidate evaluated at each
# point and combined as Eq. (3.4) prints), counted by the oracle's operation-counting
# build on a periodic grid, where no halo is counted.  The CPU suite checks these numbers
# against that build.  A kernel whose algebra needs fewer operations than the oracle's
# (the GPU combines the candidates' coefficients before evaluating, and projects p0's
# coefficients instead of the data) can reach a fraction above 1 on this basis.
ALG_FLOPS = {
    "gr": {"traces": 8126.0, "limiter": 285.0, "weak_moments": 351.0, "gradients": 6516.0,
           "face_fluxes": 846.0, "balances": 736.0, "alpha": 12.0, "stage_update": 151.0 / 3.0},
    "dr": {"traces": 12905.0, "limiter": 285.0, "weak_moments": 0.0, "gradients": 609.0,
           "face_fluxes": 846.0, "balances": 736.0, "alpha": 12.0, "stage_update": 151.0 / 3.0},
}
# the phases each kernel of the FP64 GR operator performs
KERNEL_PHASES = {"cons_recon": ("traces", "limiter"), "grad_recon": ("gradients",),
                 "flux": ("face_fluxes", "alpha"), "assemble": ("balances",)}
# the FP64 operations the mixed path keeps per interior cell-stage, counted from its
# expressions as the oracle's counter counts (an add or a multiply each): the average
# balances from the FP64 face sums (4 variables x 2 differences, 2 products and a sum),
# the averages' stage update (4 x (2 + 5 + 5) / 3 over the three stages) and the
# admissibility test (6).  The moments update in FP32, and the limiter's FP64 route runs
# only for the cells the FP32 filter cannot clear (the run's pp_percent).
MIXED_FP64_PER_CELL_STAGE = 4 * 5 + 4 * (2 + 5 + 5) / 3.0 + 6

# FP64 flops the kernels themselves execute per processed cell (DADD + DMUL + 2 DFMA,
# counted by ncu on the 256x128 shock tube): the pipe-efficiency view beside the
# algorithmic one
EXECUTED_FLOPS_PER_CELL = {"cons_recon": 5011.0, "grad_recon": 3108.0}

# algorithmic bytes per cell-stage of the unfused residual and stage update: the
# residual reads 12 state values and writes 12 residual values and 8 modified moments,
# the stage update reads 12 stage, 12 base and 20 residual/moment values and writes 12
ALG_BYTES_PER_CELL_STAGE = 8 * ((12 + 20) + (12 + 12 + 20 + 12))

# DRAM bytes of one cons_recon (k_cons<double>) launch on the 1024x512 shock tube,
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture of the current
# k_cons; valid for that grid only
K_CONS_TRAFFIC = {(1024, 512): 56591616 + 533202688}


def MEASURED_HBM_GBS():
    """the HBM copy bandwidth of MEASURED_PEAKS.json (written on the B300s), or None"""
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return None


def alg_flops(scheme, phases=None):
    f = ALG_FLOPS[scheme]
    return sum(f[p] for p in (phases or f))


def k_cons_algorithmic_bytes(nx, ny):
    """what one cons_recon launch must move: the 12 state planes read once (96 B) and
    89 output planes (traces, volume values, cell means, limiter factors: 712 B) per
    processed cell of the interior grown by 3, plus the 8 modified-moment planes (64 B)
    per interior cell"""
    return 808 * (nx + 6) * (ny + 6) + 64 * nx * ny


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hweno", choices=["hweno", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fd-directions", type=int, default=4)
    ap.add_argument("--adj-n", type=int, default=512)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-dr", action="store_true")
    ap.add_argument("--fd-plain", action="store_true",
                    help="adjoint: one central difference per direction instead of the Richardson pair")
    ap.add_argument("--no-metric-children", action="store_true",
                    help="skip the child processes that measure the adjoint, the ensemble and the colliding streams")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the child process that measures the 1D solver and the open faces")
    ap.add_argument("--mms-meshes", default="40,80,120,160")
    ap.add_argument("--mms-schemes", default="gr,dr")
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--workload", default="shock_tube",
                    choices=["shock_tube", "ensemble", "smooth_periodic", "colliding_streams", "taylor_green",
                             "adjoint", "mms", "next"],
                    help="shock_tube is the headline line; the others print their own line")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running"""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args, backend=None):
    """Ranks from the torchrun environment; for world size > 1 a process group (NCCL,
    one GPU per rank, when CUDA is present, else gloo; or the backend given)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def replica_value(ws, cells, stages, ms_max):
    """whole-job throughput of ws replicas that each advanced `cells` cells through
    `stages` RK stages, timed by the slowest rank: Gcell-RK-stage/s"""
    return ws * cells * stages / (ms_max * 1e-3) / 1e9


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_step_rate(case, q, steps=1):
    """FP64 CPU oracle: cell-stages per second over `steps` SSP-RK3 steps, the elapsed
    time, the final state and the step sizes taken."""
    from oracle import oracle as O
    cfg = O.make_cfg(**case.params())
    O.build()
    t0 = time.perf_counter()
    qq, dts = q, []
    for _ in range(steps):
        qq, st = O.step(cfg, qq)
        dts.append(st["dt"])
    el = time.perf_counter() - t0
    return case.nx * case.ny * 3.0 * steps / el, el, qq, dts


def oracle_single_thread(nx=256, ny=128):
    """The oracle on one host thread (a child process with OMP_NUM_THREADS=1): one
    SSP-RK3 step of the shock tube at nx x ny, in Gcell-RK-stage/s."""
    code = ("import json, sys; sys.path.insert(0, %r)\n"
            "from paper_2608_10569_b300 import inputs as I\n"
            "import bench\n"
            "case, q = I.shock_tube(%d, %d)\n"
            "rate, el, _, _ = bench.oracle_step_rate(case, q)\n"
            "print(json.dumps({'value': rate / 1e9, 'seconds': el}))\n" % (HERE, nx, ny))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        r = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the baseline is context
        return {"error": str(e)[:200]}
    return {"value": r["value"], "unit": METRIC, "cores": 1,
            "sample": "one SSP-RK3 step of the %dx%d shock tube, %.1f s" % (nx, ny, r["seconds"])}


def state_errors(q, ref, gamma):
    """Errors of q against ref: relative L1 and L-infinity of the density average plane,
    and the worst plane, every plane (average and moments) of a conserved variable
    measured against that variable's scale in ref (max rho; max(|rho u|, |rho v|,
    rho c) for both momenta; max E), L1 as the mean absolute error over that scale"""
    q, ref = np.asarray(q), np.asarray(ref)
    rho, m, n, E = ref[0], ref[1], ref[2], ref[3]
    p = (gamma - 1.0) * (E - 0.5 * (m * m + n * n) / rho)
    mom = max(np.abs(m).max(), np.abs(n).max(), (rho * np.sqrt(np.maximum(gamma * p / rho, 0.0))).max())
    scale = [np.abs(rho).max(), mom, mom, np.abs(E).max()]
    d = np.abs(q - ref).reshape(12, -1)
    l1 = [d[k].mean() / scale[k % 4] for k in range(12)]
    linf = [d[k].max() / scale[k % 4] for k in range(12)]
    return {"rel_l1_rho": float(d[0].sum() / np.abs(rho).sum()), "rel_linf_rho": float(d[0].max() / np.abs(rho).max()),
            "max_plane_l1": float(max(l1)), "max_plane_linf": float(max(linf))}


def cpu_threads():
    """the host threads the oracle's OpenMP loops use: OMP_NUM_THREADS, else the CPUs
    this process may run on"""
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else len(os.sched_getaffinity(0))


REFERENCE_BUDGET_S = 180.0


def workload_config(nx, ny, ws):
    """the static description of the headline workload, the same in both arms"""
    return {"workload": WORKLOAD, "nx": nx, "ny": ny, "cells": nx * ny, "stages_per_step": 3,
            "l2": "inputs larger than L2 (~1.5 GB state and scratch per step)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def run_reference(args):
    """the oracle on the host cores, on the headline's own workload: --warmup and --steps
    SSP-RK3 steps, each of the full 1024x512 shock tube when all of them fit
    REFERENCE_BUDGET_S at the first step's pace, else each of the largest box of its
    cells (the domain halved in both directions until they fit) that does"""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from paper_2608_10569_b300 import inputs as I
    from oracle import oracle as O
    O.build()
    nx, ny = args.nx, args.ny
    total = args.steps + args.warmup
    while True:
        case, q = I.shock_tube(nx, ny)
        cfg = O.make_cfg(**case.params())
        t0 = time.perf_counter()
        qq, _ = O.step(cfg, q)
        first = time.perf_counter() - t0
        if first * total <= REFERENCE_BUDGET_S or nx <= 64:
            break
        nx, ny = nx // 2, ny // 2
    for _ in range(args.warmup - 1):
        qq, _ = O.step(cfg, qq)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        qq, _ = O.step(cfg, qq)
    el = time.perf_counter() - t0
    val = nx * ny * 3.0 * args.steps / el / 1e9
    sample = "each step: one SSP-RK3 step of the shock tube at %dx%d (%s)" % (
        nx, ny, "the full workload" if nx == args.nx else "%d/%d of its cells" % (nx * ny, args.nx * args.ny))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.nx, args.ny, ws),
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_error(params, q, nsteps=10):
    """Relative L1 and L-infinity error of the mixed path's density against the FP64
    path after nsteps steps from q, both at the FP64 path's step sizes."""
    import torch
    from paper_2608_10569_b300 import hweno
    s64 = hweno.Solver(params, precision="fp64")
    s32 = hweno.Solver(params, precision="mixed")
    s64.set_state(torch.from_numpy(q).cuda())
    s32.set_state(torch.from_numpy(q).cuda())
    try:
        for _ in range(nsteps):
            dt, _ = s64.step()
            s32.step(dt)
        r64, r32 = s64.get_state()[0], s32.get_state()[0]
        d = (r32 - r64).abs()
        return {"rel_l1_rho_vs_fp64": float(d.sum() / r64.abs().sum()),
                "rel_linf_rho_vs_fp64": float(d.max() / r64.abs().max()), "steps": nsteps}
    except hweno.HwenoError as e:
        return {"error": str(e)}
    finally:
        s64.close()
        s32.close()


def run_ensemble(args):
    """64 periodic Taylor-Green cases (sides 128..1024, Re 1e2..1e4), mixed precision,
    advanced together by the batched solver: one graph replay per SSP-RK3 step."""
    import torch
    from paper_2608_10569_b300 import hweno, inputs as I
    ens = I.ensemble(64)
    cells = sum(c.nx * c.ny for c, _ in ens)
    stream = torch.cuda.Stream()
    b = hweno.Batch([c.params() for c, _ in ens], precision="mixed", stream=stream)
    for view, (case, q) in zip(b.cases, ens):
        view.set_state(q)
    chosen = b.autotune()
    b.step(args.warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    n0 = b.launch_count()
    clocks = ClockSampler(0)
    clocks.start()
    ev0.record(stream)
    rej = b.step(args.steps)
    ev1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = b.launch_count() - n0
    pp = sum(v.diag()["pp_active"] for v in b.cases)
    b.close()
    # the batched mixed path equals single mixed solvers bit for bit (tested), so one
    # case of each side states the ensemble's error against FP64
    acc, seen = [], set()
    for case, q in ens:
        if case.nx not in seen:
            seen.add(case.nx)
            acc.append(dict(mixed_error(case.params(), q, nsteps=args.steps), side=case.nx))
    errs = [a for a in acc if "error" not in a]
    line = {"metric": METRIC, "value": cells * 3.0 * args.steps / (ms * 1e-3) / 1e9, "unit": METRIC,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": "ensemble of 64 periodic Taylor-Green cases, sides 128-1024, "
                                   "Re 1e2-1e4, batched (one graph per step)", "cells": cells,
                       "autotuned_shapes": chosen, "rejected_case_steps": rej},
            "gpu_launches": launches, "clocks": clk,
            "pp_active_cell_stages": pp,
            "accuracy": {"rel_l1_rho_vs_fp64": max(a["rel_l1_rho_vs_fp64"] for a in errs) if errs else None,
                         "rel_linf_rho_vs_fp64": max(a["rel_linf_rho_vs_fp64"] for a in errs) if errs else None,
                         "sample": "one case of each side, mixed vs FP64 over the run's steps at the FP64 "
                                   "step sizes",
                         "cases": acc}}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Gradient of J = 1/2 sum (rho(T) - rho*)^2 dx dy after --steps SSP-RK3 steps of the
    Taylor-Green flow (512^2, Re 1600, Mach 0.3), checkpoints every 20 steps, with
    respect to the initial state and mu = 1/Re; time of the backward pass over the
    forward pass, and central-difference checks on seeded directions (the step sizes of
    the forward run are reused)."""
    import torch
    from paper_2608_10569_b300 import hweno, inputs as I
    steps = args.steps
    case, q = I.adjoint_taylor_green(args.adj_n)
    params = case.params()
    target = torch.from_numpy(I.adjoint_target(case)).cuda()
    area = case.dx * case.dy

    def J(qT):
        return 0.5 * ((qT[0] - target) ** 2).sum() * area

    # warm-up: library load, allocation paths and caches on a short rollout
    qw = torch.from_numpy(q).cuda().requires_grad_(True)
    muw = torch.tensor(1.0 / case.Re, dtype=torch.float64, device="cuda", requires_grad=True)
    J(hweno.rollout(qw, muw, params, nsteps=max(args.warmup, 2), ckpt=20)).backward()
    q0 = torch.from_numpy(q).cuda().requires_grad_(True)
    mu = torch.tensor(1.0 / case.Re, dtype=torch.float64, device="cuda", requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qT = hweno.rollout(q0, mu, params, nsteps=steps, ckpt=20)
    loss = J(qT)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g0 = q0.grad.cpu().numpy()
    gmu = float(mu.grad)
    s = hweno.Solver(params)
    s.set_state(q.copy())
    dts = [s.step()[0] for _ in range(steps)]
    s.close()

    def rho_T(qi, Re):
        p = dict(params)
        p["Re"] = Re
        sv = hweno.Solver(p)
        sv.set_state(torch.from_numpy(qi).cuda())
        for dt in dts:
            sv.step(dt)
        out = sv.get_state()[0].clone()
        sv.close()
        return out

    def dJ(ra, rb):  # J(a) - J(b) without the cancellation of two nearly equal sums
        return float(0.5 * ((ra - rb) * (ra + rb - 2.0 * target)).sum() * area)

    def rich(f, h):  # central differences at h and h/2, Richardson-extrapolated
        d1 = dJ(f(h), f(-h)) / (2 * h)
        if args.fd_plain:
            return d1
        d2 = dJ(f(h / 2), f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    rng = np.random.default_rng(16)
    scale = np.abs(q).reshape(12, -1).max(1)[:, None, None]
    errs = []
    for _ in range(args.fd_directions):
        v = rng.normal(size=q.shape) * scale
        fd = rich(lambda e: rho_T(q + e * v, case.Re), 1e-7)
        errs.append(abs((g0 * v).sum() - fd) / abs(fd))
    mu0 = 1.0 / case.Re
    fdmu = rich(lambda e: rho_T(q, 1.0 / (mu0 + e)), 0.02 * mu0)
    line = {"metric": "adjoint/forward time ratio", "workload": "adjoint Taylor-Green %d^2, Re 1600, Mach 0.3, "
            "%d SSP-RK3 steps, checkpoints every 20" % (args.adj_n, steps),
            "forward_s": t1 - t0, "backward_s": t2 - t1, "value": (t2 - t1) / (t1 - t0), "unit": "ratio",
            "higher_is_better": False, "dtype": "f64", "J": float(loss),
            "fd_directions": args.fd_directions, "fd_max_rel_err": max(errs) if errs else None,
            "fd_rel_errs": [float(e) for e in errs],
            "fd": "central differences at h = 1e-7 of the state scale per plane%s, the forward's step sizes "
                  "frozen" % ("" if args.fd_plain else ", Richardson-extrapolated with h/2"),
            "dJ_dmu": gmu, "mu_fd_rel_err": abs(gmu - fdmu) / abs(fdmu)}
    print(json.dumps(line), flush=True)


def run_mms(args):
    """Example 5.2 on the GPU: the manufactured-source convergence study of Table 5.2 for
    HWENO-GR and HWENO-DR.  Each mesh runs from the exact initial moments to T = 0.1
    under the Sec. 5 step rule (dt = b Re h^2 here); the errors are those of the density
    cell averages against the exact solution's, L-infinity and L1 (mean over the unit
    square), with the orders between successive meshes and the step rates."""
    import torch
    from paper_2608_10569_b300 import hweno, inputs as I
    meshes = [int(m) for m in args.mms_meshes.split(",")]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for scheme in args.mms_schemes.split(","):
        rows = []
        for n in meshes:
            case, q = I.manufactured(n, 0.0)
            _, qex = I.manufactured(n, case.t_end)
            s = hweno.Solver(dict(case.params(), scheme=scheme))
            s.set_state(torch.from_numpy(q).cuda())
            torch.cuda.synchronize()
            ev0.record(stream)
            t, steps = s.advance(case.t_end)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            err = s.get_state().cpu().numpy()[0] - qex[0]
            s.close()
            row = {"n": n, "steps": steps, "t": t, "linf": float(np.abs(err).max()),
                   "l1": float(np.abs(err).mean()), "s": ms * 1e-3,
                   "Gcell_stage_per_s": n * n * 3.0 * steps / (ms * 1e-3) / 1e9}
            if rows:
                r = n / rows[-1]["n"]
                row["order_linf"] = float(np.log(rows[-1]["linf"] / row["linf"]) / np.log(r))
                row["order_l1"] = float(np.log(rows[-1]["l1"] / row["l1"]) / np.log(r))
            rows.append(row)
            print(json.dumps({"scheme": scheme, **row}), file=sys.stderr, flush=True)
        out[scheme] = rows
    line = {"metric": "Example 5.2 errors and orders", "workload": "manufactured source, [0,1]^2 periodic, "
            "Re 100, Pr 0.72, T = 0.1, dt = min(CFL h / alpha*, b Re h^2)", "dtype": "f64", "data": "synthetic",
            "results": out}
    print(json.dumps(line), flush=True)


def pp_pct(d):
    """limiter activations as a percentage of the cell-stages evaluated (Table 5.3's
    PP-limiter column)"""
    return 100.0 * d["pp_active"] / d["cell_stages"] if d["cell_stages"] > 0 else None


def _bounded_run(s, t_end, max_steps, wall_s):
    """rule steps until t_end, max_steps, wall_s seconds or the first failed step"""
    import torch
    from paper_2608_10569_b300 import hweno
    t0 = time.perf_counter()
    status, beta = 0, []
    while True:
        d = s.diag()
        if d["t"] >= t_end or d["steps"] >= max_steps or time.perf_counter() - t0 > wall_s:
            break
        try:
            s.step()
        except hweno.HwenoError as e:
            status = e.code
            break
        beta.append(s.diag()["beta_max"])
    torch.cuda.synchronize()
    d = s.diag()
    return {"status": status, "t": d["t"], "steps": d["steps"], "rejected": d["rejected"], "pp_percent": pp_pct(d),
            "dt_last": d["dt_last"], "beta_max_first": beta[0] if beta else None,
            "beta_max_last": beta[-1] if beta else None,
            # the range the paper's beta_max figure describes, over the steps taken
            "beta_max_percentiles_10_50_90": [float(v) for v in np.percentile(beta, [10, 50, 90])] if beta else None,
            "wall_s": time.perf_counter() - t0}


def run_next(args):
    """The widened rows on the GPU, a JSON line after each block (the last one complete):
    - the 1D solver (one thread block per problem): an ensemble of 4 x 148 periodic
      problems of 256 cells, 50 steps each, for the throughput of a full GPU; Example 5.4
      (the double rarefaction, 200 cells, T = 0.6) for both schemes; and, last,
      Example 5.1's convergence study, Table 5.1's seven meshes for both schemes in one
      launch to T = 0.1, with the density errors, orders and step rates;
    - the inflow and outflow faces: the shock tube's 1024 x 512 box with open faces
      (FP64 step rate next to the headline's wall-bounded one); Example 5.7 (Sedov 2D,
      160^2, T = 1) and Example 5.9 (Mach 2000, 640 x 320, T = 0.001) under the Sec. 5
      rule until T or the first step that stays inadmissible, bounded in steps and
      wall time (25 s each), for both schemes, and Sedov once more with Remark 3.1's ablation (the
      linear weights in the gradient reconstruction)."""
    import torch
    from paper_2608_10569_b300 import hweno, inputs as I
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record(stream)
        r = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return r, ev0.elapsed_time(ev1)

    out = {"metric": "widened rows", "dtype": "f64", "data": "synthetic"}

    def snapshot():
        # the rows so far, one complete line per block, so that a time limit keeps them
        print(json.dumps(dict(out, partial=True)), flush=True)

    # ---- 1D: an ensemble filling the GPU ------------------------------------------
    for scheme in ("gr", "dr"):
        nprob, n, steps = 4 * 148, 256, 50
        params, states = [], []
        for k in range(nprob):
            p, q = I.random_smooth_1d(n, seed=1000 + k)
            params.append(dict(p, scheme=scheme))
            states.append(torch.from_numpy(q).cuda())
        res, ms = timed(lambda: hweno.advance1d(params, states, 0.0, 1e9, max_steps=steps, stream=stream))
        done = sum(r["steps"] for r in res)
        out["ensemble1d_" + scheme] = {"problems": nprob, "cells": n, "steps": steps, "ms": ms,
                                       "failed": sum(1 for r in res if r["status"] != 0),
                                       "Gcell_stage_per_s": 3.0 * n * done / (ms * 1e-3) / 1e9}
        snapshot()

    # ---- 1D: Example 5.4, the double rarefaction, both schemes in one launch -------------
    p, q = I.double_rarefaction(200)
    params = [dict(p, scheme="gr"), dict(p, scheme="dr")]
    states = [torch.from_numpy(q).cuda() for _ in params]
    res, ms = timed(lambda: hweno.advance1d(params, states, 0.0, 0.6, max_steps=100000, stream=stream))
    for r in res:  # Table 5.3's PP-limiter column: activations over the cell-stages evaluated
        r["pp_percent"] = 100.0 * r["pp_active"] / (3.0 * r["steps"] * p["n"]) if r["steps"] else None
    out["example_5_4_200"] = {"launches": 1, "ms": ms, "T": 0.6, "gr": res[0], "dr": res[1],
                              "table_5_3_pp_percent": {"gr": 8.69e-4, "dr": 1.18e-2},
                              "min_rho": [float(st.cpu().numpy()[0].min()) for st in states]}
    snapshot()

    # ---- open faces: the shock tube's box --------------------------------------------
    case, q = I.open_shock_tube(args.nx, args.ny)
    s = hweno.Solver(case.params(), precision="fp64", stream=stream)
    s.set_state(torch.from_numpy(q).cuda())
    for _ in range(args.warmup):
        s.step()
    s.profile(True)
    _, ms = timed(lambda: [s.step() for _ in range(args.steps)])
    prof = s.profile_read()
    s.profile(False)
    out["open_shock_tube"] = {"nx": case.nx, "ny": case.ny, "steps": args.steps, "ms_per_step": ms / args.steps,
                              "Gcell_stage_per_s": case.nx * case.ny * 3.0 * args.steps / (ms * 1e-3) / 1e9,
                              "rejected": s.diag()["rejected"], "pp_percent": pp_pct(s.diag()),
                              "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}}
    s.close()
    snapshot()
    # ---- open faces: Examples 5.7 and 5.9 ----------------------------------------------
    for name, make, cap in (("sedov_2d_160", lambda: I.sedov_2d(160), 400),
                            ("mach2000_640x320", lambda: I.mach2000(640, 320), 1500)):
        for scheme in ("gr", "dr"):
            case, q = make()
            s = hweno.Solver(dict(case.params(), scheme=scheme), precision="fp64", stream=stream)
            s.set_state(torch.from_numpy(q).cuda())
            out["%s_%s" % (name, scheme)] = dict(_bounded_run(s, case.t_end, cap, 25.0), T=case.t_end)
            s.close()
            snapshot()
    # Remark 3.1's ablation: the linear weights in the gradient reconstruction
    case, q = I.sedov_2d(160)
    s = hweno.Solver(dict(case.params(), linear_grad=True), precision="fp64", stream=stream)
    s.set_state(torch.from_numpy(q).cuda())
    out["sedov_2d_160_gr_linear_grad"] = dict(_bounded_run(s, case.t_end, 400, 25.0), T=case.t_end)
    s.close()
    snapshot()
    # ---- 1D: Example 5.1's study in one launch ------------------------------------
    # at the literal viscous cap b = 0.001 (dt = 0.1 h^2: 78,400 steps at 280 cells, whose
    # FP64 round-off floors the errors near 1e-11) and at b = 0.01 (ten times fewer steps)
    meshes = (40, 80, 120, 160, 200, 240, 280)
    params, states, exact, keys = [], [], [], []
    for b_visc in (1e-3, 1e-2):
        for scheme in ("gr", "dr"):
            for n in meshes:
                p, q = I.manufactured_1d(n, 0.0)
                params.append(dict(p, scheme=scheme, b_visc=b_visc))
                states.append(torch.from_numpy(q).cuda())
                exact.append(I.manufactured_1d(n, 0.1)[1][0])
                keys.append("%s_b%g" % (scheme, b_visc))
    res, ms = timed(lambda: hweno.advance1d(params, states, 0.0, 0.1, stream=stream))
    rows = {k: [] for k in dict.fromkeys(keys)}
    cell_stages = 0.0
    for p, st, ex, r, key in zip(params, states, exact, res, keys):
        err = st.cpu().numpy()[0] - ex
        row = {"n": p["n"], "steps": r["steps"], "status": r["status"], "t": r["t"],
               "linf": float(np.abs(err).max()), "l1": float(np.abs(err).mean())}
        prev = rows[key]
        if prev:
            ratio = row["n"] / prev[-1]["n"]
            row["order_linf"] = float(np.log(prev[-1]["linf"] / row["linf"]) / np.log(ratio))
            row["order_l1"] = float(np.log(prev[-1]["l1"] / row["l1"]) / np.log(ratio))
        prev.append(row)
        cell_stages += 3.0 * r["steps"] * p["n"]
    out["example_5_1"] = {"launches": 1, "problems": len(params), "ms": ms, "rows": rows,
                          "Gcell_stage_per_s": cell_stages / (ms * 1e-3) / 1e9,
                          "note": "one block per problem; the 280-cell problems at b = 0.001 (78,400 steps) "
                                  "bound the launch"}
    print(json.dumps(out), flush=True)


def child_line(argv, timeout):
    """bench.py with argv in a child process (its own CUDA context), bounded in time: its
    last JSON line, or the error; a failure there never reaches the headline measurement"""
    cmd = [sys.executable, os.path.join(HERE, "bench.py")] + list(argv)

    def last_line(text):
        for line in reversed((text or "").strip().splitlines()):
            try:
                return json.loads(line)
            except ValueError:
                continue
        return {}

    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
        out = last_line(r.stdout)
        if r.returncode != 0:
            out["error"] = "exit %d: %s" % (r.returncode, r.stderr.strip()[-300:])
        return out
    except subprocess.TimeoutExpired as e:
        so = e.stdout.decode() if isinstance(e.stdout, bytes) else e.stdout
        return dict(last_line(so), error="time limit of %d s reached; the rows above are those completed" % timeout)
    except Exception as e:
        return {"error": str(e)[:300]}


def next_rows_child(args):
    """run_next in a child process, bounded to 360 s"""
    return child_line(["--workload", "next", "--steps", "3", "--warmup", "1"], 360)


def metric_children(args):
    """the rest of the metric, each in a child process: the 512^2 adjoint (200 steps,
    checkpoints every 20, forward and backward times, central differences on 16 seeded
    directions), the ensemble (64 cases, 100 batched mixed steps, the worst case
    against FP64), the colliding streams (2048^2) and the coarse rows of Example 5.2's
    convergence study (GR and DR at 40^2 and 80^2, about 20 s)"""
    return {
        "adjoint": child_line(["--workload", "adjoint", "--steps", "200", "--warmup", "2", "--fd-directions", "16",
                               "--fd-plain"], 420),
        "ensemble": child_line(["--workload", "ensemble", "--steps", "100", "--warmup", "3"], 300),
        "colliding_streams": child_line(["--workload", "colliding_streams", "--steps", "3", "--warmup", "1"], 300),
        "mms": child_line(["--workload", "mms", "--mms-meshes", "40,80", "--mms-schemes", "gr,dr"], 120),
    }


def run_single(args):
    """the smooth periodic flow, the colliding streams and the Taylor-Green flow on one
    solver: FP64 and mixed step rates with the mixed path's error against FP64 (the
    colliding streams, whose limited states make the step rule restart ~20 times per
    step, report residual evaluations as well, and their mixed handle runs the FP64
    operator: its internal energy is 7.5e-7 of the total)"""
    import torch
    from paper_2608_10569_b300 import hweno, inputs as I
    if args.workload == "smooth_periodic":
        case, q = I.smooth_periodic(64)
    elif args.workload == "taylor_green":
        case, q = I.adjoint_taylor_green(512)
    else:
        case, q = I.colliding_streams(2048)
    cells = case.nx * case.ny
    out, final = {}, {}
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for prec in ("fp64", "mixed"):
        s = hweno.Solver(case.params(), precision=prec)
        s.set_state(torch.from_numpy(q).cuda())
        try:
            out[prec] = _time_single(args, s, cells, stream, ev0, ev1)
            final[prec] = s.get_state().cpu().numpy()
        except hweno.HwenoError as e:
            out[prec] = {"error": str(e)}
        s.close()
    if "error" not in out.get("mixed", {}) and args.workload != "colliding_streams":
        out["mixed"]["accuracy"] = mixed_error(case.params(), q)
    elif "fp64" in final and "mixed" in final:
        d = np.abs(final["mixed"][0] - final["fp64"][0])
        out["mixed"]["accuracy"] = {"rel_l1_rho_vs_fp64": float(d.sum() / np.abs(final["fp64"][0]).sum()),
                                    "rel_linf_rho_vs_fp64": float(d.max() / np.abs(final["fp64"][0]).max()),
                                    "steps": args.warmup + args.steps}
    line = {"metric": METRIC, "unit": METRIC, "workload": args.workload, "cells": cells,
            "steps": args.steps, "warmup": args.warmup, "results": out}
    print(json.dumps(line), flush=True)


def _time_single(args, s, cells, stream, ev0, ev1):
    import torch
    out = {}
    if args.workload == "colliding_streams":
        rhs, vh = s.residual()
        for _ in range(args.warmup):
            s.residual(rhs, vh)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            s.residual(rhs, vh)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        out.update({"Gcell_residual_per_s": cells * args.steps / (ms * 1e-3) / 1e9,
                    "ms_per_residual": ms / args.steps})
    for _ in range(args.warmup):
        s.step()
    d0 = s.diag()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        s.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    d = s.diag()
    out.update({"value": cells * 3.0 * args.steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / args.steps,
                "rejected": d["rejected"] - d0["rejected"], "fp64_steps": d["fp64_steps"] - d0["fp64_steps"],
                "max_kinetic_share": d["max_kinetic_share"], "t_reached": d["t"], "pp_percent": pp_pct(d),
                "min_rho": d["min_rho"]})
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "mms":
        return run_mms(args)
    if args.workload == "next":
        return run_next(args)
    if args.workload != "shock_tube":
        return run_single(args)
    import torch
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2608_10569_b300 import hweno, inputs as I

    case, q = I.shock_tube(args.nx, args.ny)
    cells = case.nx * case.ny
    stream = torch.cuda.current_stream()
    qd = torch.from_numpy(q).cuda()

    # ---- FP64 path, device-resident ------------------------------------------------
    s = hweno.Solver(case.params(), precision="fp64", stream=stream)
    s.set_state(qd)
    for _ in range(args.warmup):
        s.step()
    peak64 = s.measure_peak(0)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    s.profile(True)
    n0 = s.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    rejected = 0
    for _ in range(args.steps):
        _, rej = s.step()
        rejected += rej
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = s.launch_count() - n0
    clk = clocks.stop()
    prof = s.profile_read()
    s.profile(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ws, ms)
    stages = 3.0 * args.steps
    value = replica_value(ws, cells, stages, ms_max)
    q_fp64 = s.get_state().cpu().numpy()
    t_reached = s.diag()["t"]
    pp_percent = pp_pct(s.diag())

    # dominant kernel of the operator and its roofline against the FP64 FMA peak, on the
    # algorithmic flop count; the whole step on the same basis
    dom = max((k for k in prof if k != "rk_update"), key=lambda k: prof[k][1])
    n_l, tot_ms = prof[dom]
    roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": peak64,
            "peak_source": "measured FP64 FMA peak (hweno_measure_peak, this run)",
            "flops_basis": "algorithmic: the FP64 oracle's distinct operations per interior cell "
                           "(its operation-counting build), not the kernel's own count",
            "launches": n_l, "mean_launch_ms": tot_ms / max(n_l, 1),
            "share_of_step": tot_ms / ms if ms > 0 else None,
            "traffic": K_CONS_TRAFFIC.get((case.nx, case.ny)) if dom == "cons_recon" else None,
            "algorithmic_bytes": k_cons_algorithmic_bytes(case.nx, case.ny) if dom == "cons_recon" else None}
    if dom in KERNEL_PHASES and n_l:
        fpc = alg_flops("gr", KERNEL_PHASES[dom])
        launch_s = tot_ms / n_l * 1e-3
        achieved = fpc * cells / launch_s / 1e12
        roof.update({"achieved": achieved, "frac": achieved / peak64, "flops_per_cell": fpc})
        if dom in EXECUTED_FLOPS_PER_CELL:
            ex = EXECUTED_FLOPS_PER_CELL[dom] * cells / launch_s / 1e12
            roof.update({"executed_flops_per_cell": EXECUTED_FLOPS_PER_CELL[dom], "executed_achieved": ex,
                         "executed_frac": ex / peak64})
    else:
        roof.update({"achieved": None, "frac": None, "flops_per_cell": None})
    step_flops = alg_flops("gr")
    step_achieved = step_flops * cells * stages / (ms * 1e-3) / 1e12
    roof["step"] = {"flops_per_cell_stage": step_flops, "achieved": step_achieved, "frac": step_achieved / peak64,
                    "per_kernel_frac": {k: alg_flops("gr", ph) * cells / (prof[k][1] / prof[k][0] * 1e-3) / 1e12
                                        / peak64 for k, ph in KERNEL_PHASES.items() if prof.get(k, (0,))[0]}}
    kernel_ms = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}

    # ---- end to end through the C ABI with host buffers ---------------------------
    e2e = None
    hq = torch.from_numpy(q.copy()).pin_memory()
    hout = torch.empty_like(hq).pin_memory()
    s.set_state(hq)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_state(hq)
        s.step()
        s.get_state(hout)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    el = max_over_ranks(ws, el)
    nbytes = q.nbytes
    e2e = {"value": ws * cells * stages / el / 1e9, "unit": METRIC, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    s.close()

    # ---- mixed precision on the same steps ----------------------------------------
    mixed = None
    if not args.no_mixed:
        m = hweno.Solver(case.params(), precision="mixed", stream=stream)
        m.set_state(qd)
        for _ in range(args.warmup):
            m.step()
        peak32 = m.measure_peak(1)
        m.set_state(qd)
        torch.cuda.synchronize()
        m.profile(True)
        ev0.record(stream)
        for _ in range(args.steps):
            m.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        mprof = m.profile_read()
        m.profile(False)
        mms = max_over_ranks(ws, ev0.elapsed_time(ev1))
        qm = m.get_state().cpu().numpy()
        # L1 error against the FP64 path after the same number of steps from the same state
        # (the FP64 path matches the FP64 oracle to round-off)
        s64 = hweno.Solver(case.params(), precision="fp64", stream=stream)
        s64.set_state(qd)
        for _ in range(args.steps):
            s64.step()
        q64 = s64.get_state().cpu().numpy()
        s64.close()
        l1 = float(np.abs(qm[0] - q64[0]).sum() / np.abs(q64[0]).sum())
        linf = float(np.abs(qm[0] - q64[0]).max() / np.abs(q64[0]).max())
        # the mixed step's roofline on the same algorithmic basis: the oracle's operations
        # less those the mixed path keeps in FP64 against the measured FP32 FMA peak, those
        # against the FP64 one, the unfused bytes against the HBM bandwidth; the slowest
        # bounds the cell-stage rate
        f64 = MIXED_FP64_PER_CELL_STAGE
        f32 = alg_flops("gr") - f64
        hbm = MEASURED_HBM_GBS()
        bound_rate = min(peak32 * 1e12 / f32, peak64 * 1e12 / f64,
                         hbm * 1e9 / ALG_BYTES_PER_CELL_STAGE if hbm else float("inf"))
        mrate = cells * stages / (mms * 1e-3)
        mixed_roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak32,
                      "peak_source": "measured FP32 FMA peak (hweno_measure_peak, this run)",
                      "fp32_flops_per_cell_stage": f32, "fp64_flops_per_cell_stage": f64,
                      "achieved": f32 * mrate / 1e12, "frac": f32 * mrate / 1e12 / peak32,
                      "fp64_achieved": f64 * mrate / 1e12, "fp64_frac": f64 * mrate / 1e12 / peak64,
                      "bytes_per_cell_stage": ALG_BYTES_PER_CELL_STAGE, "hbm_peak_gbs": hbm,
                      "rate_bound": bound_rate / 1e9, "frac_of_rate_bound": mrate / bound_rate}
        mixed = {"value": replica_value(ws, cells, stages, mms), "unit": METRIC,
                 "ms_per_step": mms / args.steps, "fp32_peak_tflops": peak32, "roofline": mixed_roof,
                 "rel_l1_rho_vs_fp64": l1, "rel_linf_rho_vs_fp64": linf,
                 "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in mprof.items()}}
        m.close()

    # ---- HWENO-DR, the paper's comparison scheme, on the same workload ---------------
    dr = None
    if not args.no_dr:
        d = hweno.Solver(dict(case.params(), scheme="dr"), precision="fp64", stream=stream)
        d.set_state(qd)
        for _ in range(args.warmup):
            d.step()
        torch.cuda.synchronize()
        d.profile(True)
        n0 = d.launch_count()
        ev0.record(stream)
        for _ in range(args.steps):
            d.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        dlaunch = d.launch_count() - n0
        dprof = d.profile_read()
        d.profile(False)
        dms = max_over_ranks(ws, ev0.elapsed_time(ev1))
        qdr = d.get_state().cpu().numpy()
        # both schemes took warm-up + K steps of their own step rule from the same state
        # Table 5.3 prints the CPU-time ratio T_GR / T_DR of this workload's whole run
        # (1.09) and the limiter activations of both schemes (0 %)
        dr = {"value": replica_value(ws, cells, stages, dms), "unit": METRIC, "ms_per_step": dms / args.steps,
              "time_ratio_gr_over_dr": ms_max / dms, "pp_percent": pp_pct(d.diag()),
              "gpu_launches": dlaunch, "t_reached": d.diag()["t"], "t_reached_gr": t_reached,
              "rel_l1_rho_vs_gr": float(np.abs(qdr[0] - q_fp64[0]).sum() / np.abs(q_fp64[0]).sum()),
              "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in dprof.items()}}
        dstep = alg_flops("dr")
        dach = dstep * cells * stages / (dms * 1e-3) / 1e12
        dr["step_roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak64, "flops_per_cell_stage": dstep,
                               "achieved": dach, "frac": dach / peak64}
        d.close()

    # ---- CPU baseline: the oracle on the host cores --------------------------------
    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, el, q_or, dts_or = oracle_step_rate(case, q, steps=1)
        cpu = {"value": rate / 1e9, "unit": METRIC, "cores": cpu_threads(), "kind": "oracle",
               "sample": "one SSP-RK3 step (3 stages) of the full 1024x512 workload, %.1f s" % el,
               "single_thread": oracle_single_thread()}
        # the same step on the GPU, FP64 and mixed, against the oracle's result
        parity = {"sample": "one SSP-RK3 step of the full 1024x512 workload at the oracle's step size"}
        for prec in ("fp64", "mixed"):
            sv = hweno.Solver(case.params(), precision=prec, stream=stream)
            sv.set_state(qd)
            sv.step(dts_or[0])
            parity[prec] = state_errors(sv.get_state().cpu().numpy(), q_or, case.gamma)
            sv.close()

    # ---- the rest of the metric and the widened rows, in child processes -------------
    children = {}
    if rank == 0 and ws == 1 and not args.no_metric_children:
        children = metric_children(args)
    next_rows = None
    if rank == 0 and ws == 1 and not args.no_next:
        next_rows = next_rows_child(args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(case.nx, case.ny, ws),
                "run": {"t_reached": t_reached, "rejected_steps": rejected, "pp_percent": pp_percent},
                "roofline": roof, "cpu_baseline": cpu, "parity_vs_oracle": parity, "e2e": e2e, "mixed": mixed,
                "dr": dr, **children, "next_rows": next_rows,
                "clocks": clk, "gpu_launches": launches, "kernel_ms": kernel_ms}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
