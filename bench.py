"""Benchmark of the NCS hot path on the 512x512 TV-CT workload (720 angles,
730 bins, isotropic TV, lambda 0.005, 20 seeded ellipses, 0.5% noise).

One "step" is one NCS iteration with every step of the hot path: the K^T
gather, the FFT solve with M, the primal update, the TV dual prox, the forward
projection with the data prox, and (every check_every = 10 steps) the FP64
objective reduction read back by the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is NCS iterations per second summed over
ranks (replicas: each GPU solves its own slice, no collective on the data path).
L2 is flushed (256 MiB write, untimed) before every timed step; each step is
timed with CUDA events on the plan's stream.  Also reported: time to a 1e-4
relative objective gap for NCS and PDHG on the same GPU (against the FP64
oracle's f* stored in tests/golden), per-kernel times, the roofline of the
dominant kernel, the end-to-end rate through the Python API with host buffers,
and the FP64 CPU oracle timed on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "ct512"
# NCS / PDHG parameters for this workload, tuned on the {1,3} x 10^p grid (Sec. 5)
NCS_PARAMS = dict(alpha=0.01, beta=0.01, gamma=0.0, h_probes=32)   # M's projector part by eq. (H-fan)
PDHG_PARAMS = dict(alpha=0.001, beta=0.001)
# ADMM comparator (Sec. 1.3): penalty 1/alpha, n_cg preconditioned CG steps per outer step
ADMM_PARAMS = dict(alpha=0.1, beta=0.1, n_cg=10)
ADMM_CAP = 1000                     # outer steps
CHECK_EVERY = 10
TTG_TOL = 1e-4
# the solvers stop at their own FP64 objective gap <= TTG_STOP; evaluated on FP32 state, that
# objective lies within ~1e-6 relative of the oracle's, so the 2% margin keeps the oracle's gap
# of the returned x at or below TTG_TOL
TTG_STOP = 0.98e-4
TTG_CAP = 2000                      # NCS and ADMM iteration cap of the time-to-gap runs
PDHG_CAP = 20000                    # PDHG needs ~10^4 iterations on this workload
METRIC = "time to 1e-4 rel. objective gap (512² TV-CT) vs PDHG; NCS iters/s; % HBM roofline"
# class name of the library's per-kernel timers -> kernel name in ncu's launch list
# ncu kernel names of a kernel class (the strip form of K is two kernels per launch)
NCU_KERNEL = {"joseph_gather": ["k_gather"], "joseph_fwd": ["k_fwd_strip", "k_fwd_sum"],
              "joseph_fwd_resid": ["k_fwd_strip", "k_fwd_sum"]}


def load_counters(workload, directory=None):
    """ncu counters per launch of the library's kernels for a workload, from the committed
    capture summary profiles/counters_<workload>.txt.  Each data line reads

        <ncu kernel name> <source file> <sha256 of that file> <dram bytes> <warp instructions>

    A kernel's counters are used only while its source file still has the recorded hash
    (a changed kernel gets null counters until it is captured again)."""
    import hashlib
    out = {}
    path = os.path.join(directory or os.path.join(ROOT, "profiles"), "counters_%s.txt" % workload)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return out
    for ln in lines:
        f = ln.split()
        if len(f) != 5 or ln.startswith("#"):
            continue
        name, src, sha, dram, winst = f
        try:
            cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
        except OSError:
            continue
        out[name] = {"traffic": float(dram), "warp_instr": float(winst), "current": cur == sha,
                     "source": src}
    return out


def counters_for(cnt, cls, ncu_name=None):
    """(dram bytes, warp instructions) per launch of a kernel class (summed over the kernels
    of one launch), or (None, None) when any of them has no current capture."""
    names = ncu_name or NCU_KERNEL.get(cls, [cls])
    if isinstance(names, str):
        names = [names]
    traffic = instr = 0.0
    for nm in names:
        c = cnt.get(nm)
        if not c or not c["current"]:
            return None, None
        traffic += c["traffic"]
        instr += c["warp_instr"]
    return traffic, instr


def sm_count(dev):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def load_golden(workload, seed):
    """The oracle's reference run for the workload (f*, and a fingerprint of the
    sinogram it was computed for), or None."""
    path = os.path.join(ROOT, "tests", "golden", "fstar_%s_s%d.json" % (workload, seed))
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="ncs_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def _cuda_available():
    import torch
    return torch.cuda.is_available()


def reduce_max(value, ws):
    """Max of a float over ranks (identity for one rank)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, ws):
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def make_inputs(seed, project):
    """The seeded workload: b = project(x_true) + noise (synth's recipe)."""
    import synth
    W = synth.WORKLOADS[WORKLOAD]
    pr = synth.ct_problem(seed, W["N"], W["n_angles"], W["n_det"], W["n_ellipses"], W["noise_frac"], project)
    return W, pr


def gpu_projector(plan, dev):
    """x -> K x with the library's projector (the benchmark's inputs are made on the GPU)."""
    import numpy as np
    import torch

    def project(x):
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32).ravel()).to(dev)
        return plan.apply_K(t).cpu().numpy().astype(np.float64)
    return project


# ------------------------------------------------------------------ CPU oracle leg

def oracle_rate(seed, budget_s=15.0, min_iters=2, warmup=1, max_iters=1000):
    """FP64 oracle NCS iterations per second on the host cores for a bounded
    sample of the workload (iterations from the zero state, after `warmup` untimed ones;
    at least min_iters and at most max_iters timed, stopping once the budget is spent)."""
    import numpy as np
    from oracle import circulant as oci, operators as oop, solvers as osv
    import synth
    W0 = synth.WORKLOADS[WORKLOAD]
    W, pr = make_inputs(seed, oop.projector(W0["N"], W0["n_angles"], W0["n_det"]))
    g = oop.Geometry(W["N"], W["n_angles"], W["n_det"])
    P = osv.Problem(g, pr["b"].astype(np.float64), lam=W["lam"], alpha=NCS_PARAMS["alpha"],
                    beta=NCS_PARAMS["beta"], tv=W["tv"])
    # the oracle's M with a short power iteration for the (A3) rescale: setup, not a step
    mu, _ = osv.a3_scaled_mu(P, oci.mu_table(g, P.alpha, P.beta, NCS_PARAMS["gamma"]), max_iter=3)
    Minv = osv.circulant_Minv(mu)
    st = osv.zero_state(P)
    for _ in range(max(1, warmup)):
        st = osv.ncs_step(P, st, Minv)      # warm-up (library loading, page faults)
    times = []
    t_start = time.perf_counter()
    while len(times) < min_iters or time.perf_counter() - t_start < budget_s:
        t0 = time.perf_counter()
        st = osv.ncs_step(P, st, Minv)
        if (len(times) + 1) % CHECK_EVERY == 0:
            osv.objective(P, st.x)
        times.append(time.perf_counter() - t0)
        if len(times) >= max_iters:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(rate=len(times) / sum(times), iters=len(times), seconds=sum(times), cores=cores,
                per_iter=times)


def oracle_rate_one_core(seed, budget_s=5.0):
    """oracle_rate in a child process with OMP_NUM_THREADS=1 (None if it fails)."""
    import subprocess
    code = ("import json, bench; r = bench.oracle_rate(%d, budget_s=%r); r.pop('per_iter'); print(json.dumps(r))"
            % (seed, float(budget_s)))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    per_iter_budget = max(5.0, min(150.0, 0.8 * args.steps))
    # warm-up steps (untimed, at most 5: the oracle has nothing to warm beyond the first), then
    # the K timed steps, cut short only if they would run past a few minutes
    warm = max(1, min(args.warmup, 5))
    r = oracle_rate(args.seed, budget_s=per_iter_budget, min_iters=min(args.steps, 3), warmup=warm,
                    max_iters=args.steps)
    times = r["per_iter"][: args.steps]
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": args.gpus,
        "steps": len(times), "warmup": warm, "ms_per_step": 1000.0 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 TV-CT, 720 angles x 730 bins, iso TV lambda 0.005, 20 ellipses, "
                               "0.5%% noise, seed %d" % args.seed,
                   "parallelism": "single", "l2": "n/a (host)", "ncs": NCS_PARAMS},
        "cpu_baseline": {"value": value, "unit": "it/s", "cores": r["cores"], "kind": "oracle",
                         "sample": "%d FP64 oracle NCS iterations of the 512x512 workload from zero" % len(times)},
        "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def cufft_reference(N, dev, iters=200):
    """The circulant solve done with cuFFT through torch.fft (rfft2, multiply by a
    1/mu-shaped table, irfft2 into x - Delta), timed with CUDA events on torch's
    stream; a reference for the hand-written FFT kernels only, not used by the path."""
    import torch
    r = torch.randn(N, N, device=dev)
    x = torch.randn(N, N, device=dev)
    inv = torch.rand(N, N // 2 + 1, device=dev)

    def once():
        d = torch.fft.irfft2(torch.fft.rfft2(r) * inv, s=(N, N))
        x.sub_(d)

    for _ in range(10):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        once()
    e1.record()
    torch.cuda.synchronize()
    return {"cufft_ms": e0.elapsed_time(e1) / iters,
            "what": "torch.fft.rfft2 -> complex multiply by a table -> irfft2 -> x -= Delta (cuFFT), %dx%d FP32, "
                    "L2-warm, CUDA events; ours_ms = the three hand-written FFT kernels per iteration" % (N, N)}


def admm_ttg(ncs, N, na, nd, W, b, f_star, dev, grid=False):
    """Time to the gap of the ADMM comparator (PCG inner loop preconditioned by the same
    eq. (H-fan) circulant as NCS) from zero; with grid, over alpha x n_cg as well."""
    import torch
    cfgs = [dict(ADMM_PARAMS)]
    if grid:
        cfgs += [dict(alpha=a, beta=a, n_cg=c) for a in (0.01, 0.03, 0.1, 0.3, 1.0) for c in (3, 10)
                 if (a, c) != (ADMM_PARAMS["alpha"], ADMM_PARAMS["n_cg"])]
    out = []
    x0 = None
    for c in cfgs:
        t0 = time.perf_counter()
        aplan = ncs.Plan(N, na, nd, W["lam"], c["alpha"], beta=c["beta"], tv=W["tv"], check_every=CHECK_EVERY,
                         h_probes=NCS_PARAMS["h_probes"])
        setup = _sync_ms(t0)
        x = torch.zeros(N * N, device=dev)
        rep = aplan.admm_solve(b, x, tol=TTG_STOP, max_outer=ADMM_CAP, n_cg=c["n_cg"], f_star=f_star)
        aplan.close()
        out.append(dict(c, outer=rep["iters"], time_ms=rep["time_ms"], gap=rep["gap"], status=rep["status"],
                        operator_passes=rep["iters"] * (c["n_cg"] + 2), with_setup_ms=rep["time_ms"] + setup))
        if x0 is None:
            x0 = x.cpu().numpy().astype("float64")
    return (out if grid else out[0]), x0


def projector_roofline(name, ms_per_launch, nnz, peaks, dev, counters, ncu_name=None):
    """Roofline object of a projector kernel (K or K^T): 2 flops per nonzero of K against
    the FP32 FMA peak derived from the device's SM count, 128 FP32 lanes per SM and the
    maximum SM clock ("alu"); with a current ncu capture, its DRAM traffic per launch and
    an issue roofline (warp instructions per launch over the event-timed duration against
    SMs x 4 schedulers x 1 warp instruction per cycle)."""
    if name not in ("joseph_gather", "joseph_fwd", "joseph_fwd_resid"):
        return None
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = sm_count(dev)
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12      # FMA = 2 flops
    t = ms_per_launch / 1000.0
    achieved = 2.0 * nnz / t / 1e12
    traffic, wi = counters_for(counters, name, ncu_name)
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic,
            "work": "2 flops per nonzero of K (%.4g nonzeros)" % nnz,
            "peak_kind": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % (sms, sm_mhz)}
    if wi:
        issue_peak = sms * 4 * sm_mhz * 1e6 / 1e12
        issue = wi / t / 1e12
        roof["issue"] = {"achieved": issue, "peak": issue_peak, "unit": "Twarp-inst/s", "frac": issue / issue_peak,
                         "warp_instructions_per_launch": wi,
                         "peak_kind": "%d SMs x 4 schedulers x 1 warp-instruction/cycle x %.0f MHz (derived)"
                                      % (sms, sm_mhz)}
    else:
        roof["issue"] = None
    return roof


def _sync_ms(t0):
    import torch
    torch.cuda.synchronize()
    return 1000.0 * (time.perf_counter() - t0)


def time_to_gap(args, rank, ncs, plan, W, N, na, nd, dev):
    """NCS, PDHG and ADMM-PCG from zero to the 1e-4 relative gap against the oracle's f*
    on every seed with a stored record.  Returns (summary, stops): stops[(seed, solver)] is
    the host copy of the returned x, re-evaluated by the oracle in the CPU leg."""
    import statistics
    import torch
    n = N * N
    seeds = [args.seed + rank] + [sd for sd in range(5) if sd != args.seed + rank]
    runs, stops = [], {}
    # setup, timed on the host around plan creation (synchronising): NCS builds the Joseph
    # tables, the DC entry, eq. (H-fan) over 32 probes and the (A3) power iteration; PDHG's
    # plan (pdhg_only) builds the tables and then computes lambda_max(A^T A) by power iteration
    t0 = time.perf_counter()
    nplan = ncs.Plan(N, na, nd, W["lam"], NCS_PARAMS["alpha"], beta=NCS_PARAMS["beta"], gamma=NCS_PARAMS["gamma"],
                     tv=W["tv"], check_every=CHECK_EVERY, h_probes=NCS_PARAMS["h_probes"])
    ncs_setup = _sync_ms(t0)
    t0 = time.perf_counter()
    pplan = ncs.Plan(N, na, nd, W["lam"], PDHG_PARAMS["alpha"], beta=PDHG_PARAMS["beta"], tv=W["tv"],
                     check_every=CHECK_EVERY, pdhg_only=True)
    pdhg_tables = _sync_ms(t0)
    t0 = time.perf_counter()
    lmax, _ = pplan.power_bound()
    pdhg_lmax = _sync_ms(t0)
    pdhg_setup = pdhg_tables + pdhg_lmax
    for sd in seeds:
        gold = load_golden(WORKLOAD, sd)
        if not gold:
            continue
        f_star = gold["f_star"]
        bs = torch.from_numpy(make_inputs(sd, gpu_projector(plan, dev))[1]["b"].ravel()).to(dev)
        run = {"seed": sd, "f_star": f_star, "oracle_iters": gold.get("iterations"),
               "f_star_tight": bool(gold.get("tight", False)),
               "f_star_decrease_last_1000_rel": gold["decrease_last_1000"] / abs(f_star)}
        if "b_sum" in gold:
            # the oracle's f* belongs to the sinogram made with its own K; this run's b
            # (made with the library's K) must agree to float32 rounding
            bd = bs.double()
            run["b_rel_diff"] = {"sum": abs(bd.sum().item() - gold["b_sum"]) / abs(gold["b_sum"]),
                                 "sumsq": abs((bd * bd).sum().item() - gold["b_sumsq"]) / gold["b_sumsq"]}
        xs = torch.zeros(n, device=dev)
        rep = nplan.solve(bs, xs, tol=TTG_STOP, max_iter=TTG_CAP, f_star=f_star)
        run["ncs"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        run["ncs"]["with_setup_ms"] = rep["time_ms"] + ncs_setup
        stops[(sd, "ncs")] = xs.cpu().numpy().astype("float64")
        xs.zero_()
        rep = pplan.pdhg_solve(bs, xs, tol=TTG_STOP, max_iter=PDHG_CAP, f_star=f_star)
        run["pdhg"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        run["pdhg"]["with_setup_ms"] = rep["time_ms"] + pdhg_setup
        stops[(sd, "pdhg")] = xs.cpu().numpy().astype("float64")
        adm, xa = admm_ttg(ncs, N, na, nd, W, bs, f_star, dev, args.admm_grid and not runs)
        run["admm"] = adm
        stops[(sd, "admm")] = xa
        runs.append(run)
    nplan.close()
    pplan.close()
    if not runs:
        return None, stops
    med = lambda xs_: statistics.median(xs_) if xs_ else None
    ttg = {"tol": TTG_TOL, "gpu_stop_tol": TTG_STOP, "cap": {"ncs": TTG_CAP, "pdhg": PDHG_CAP, "admm_outer": ADMM_CAP},
           "seeds": [r["seed"] for r in runs], "runs": runs,
           "setup_ms": {"ncs": ncs_setup, "pdhg": pdhg_setup, "pdhg_tables": pdhg_tables,
                        "pdhg_lambda_max": pdhg_lmax, "lambda_max_AtA": lmax,
                        "what": "host wall time of plan creation (NCS: tables, h_dc, 32 probes of eq. (H-fan), "
                                "(A3) power iteration; PDHG: a pdhg_only plan's tables + power iteration for "
                                "lambda_max(A^T A))"}}
    for solver in ("ncs", "pdhg"):
        ok = [r[solver] for r in runs if r[solver]["status"] == 0]
        ttg[solver + "_converged_gpu_objective"] = len(ok)
        ttg[solver + "_median_ms"] = med([r["time_ms"] for r in ok])
        ttg[solver + "_median_ms_with_setup"] = med([r["with_setup_ms"] for r in ok])
        ttg[solver + "_median_iters"] = med([r["iters"] for r in ok])
    adm = [r["admm"] for r in runs]
    adm = [a[0] if isinstance(a, list) else a for a in adm]
    adm_ok = [a for a in adm if a["status"] == 0]
    ttg.update({"admm": ADMM_PARAMS, "admm_converged_gpu_objective": len(adm_ok),
                "admm_median_ms": med([a["time_ms"] for a in adm_ok]),
                "admm_median_ms_with_setup": med([a["with_setup_ms"] for a in adm_ok]),
                "admm_median_outer": med([a["outer"] for a in adm_ok])})
    return ttg, stops


def oracle_check_stops(ttg, stops):
    """The CPU leg's check of the time-to-gap runs: the FP64 oracle's objective at every
    stopping point, on the sinogram the stored f* was computed for (made with the oracle's
    own K), gives the oracle gap (f(x) - f*)/|f*|.  A seed counts as converged for a solver
    only when that gap is <= the tolerance and the stored f* record is tight."""
    import numpy as np
    from oracle import operators as oop, solvers as osv
    import synth
    W = synth.WORKLOADS[WORKLOAD]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    g = oop.Geometry(N, na, nd)
    proj = oop.projector(N, na, nd)
    for r in ttg["runs"]:
        pr = synth.ct_problem(r["seed"], N, na, nd, W["n_ellipses"], W["noise_frac"], proj)
        P = osv.Problem(g, pr["b"].astype(np.float64), lam=W["lam"], alpha=1.0, beta=1.0, tv=W["tv"])
        for solver in ("ncs", "pdhg", "admm"):
            x = stops.get((r["seed"], solver))
            tgt = r[solver][0] if isinstance(r[solver], list) else r[solver]
            if x is None:
                continue
            f = osv.objective(P, x.reshape(N, N))
            tgt["oracle_f"] = f
            tgt["oracle_gap"] = (f - r["f_star"]) / abs(r["f_star"])
    for solver in ("ncs", "pdhg", "admm"):
        conv = []
        for r in ttg["runs"]:
            tgt = r[solver][0] if isinstance(r[solver], list) else r[solver]
            if "oracle_gap" in tgt and r["f_star_tight"] and tgt["status"] == 0 and tgt["oracle_gap"] <= ttg["tol"]:
                conv.append(r["seed"])
        ttg[solver + "_converged_oracle"] = len(conv)
        ttg[solver + "_converged_oracle_seeds"] = conv
    ttg["oracle_check"] = ("FP64 oracle objective at every stop on the oracle-made sinogram; a seed counts as "
                           "converged only with a tight f* record (last 1000 oracle iterations lowered f by "
                           "<= 1e-7 relative) and an oracle gap <= tol")


def oracle_check_one(ttg, workload, seed, stops):
    """The CPU leg's check of a single-seed time-to-gap line: the FP64 oracle's objective at
    each solver's stop on the sinogram the stored f* was computed for (made with the oracle's
    own K, oracle.fstar.problem); a solver counts as converged only when that gap is <= the
    tolerance, its GPU solve stopped without error and the stored f* record is tight."""
    from oracle import fstar, solvers as osv
    P, _ = fstar.problem(workload, seed)
    N = P.g.N
    for solver, x in stops.items():
        f = osv.objective(P, x.reshape(N, N))
        tgt = ttg[solver]
        tgt["oracle_f"] = f
        tgt["oracle_gap"] = (f - ttg["f_star"]) / abs(ttg["f_star"])
        ttg[solver + "_converged_oracle"] = int(bool(ttg["f_star_tight"]) and tgt["status"] == 0
                                                and tgt["oracle_gap"] <= ttg["tol"])
    ttg["oracle_check"] = ("FP64 oracle objective at every stop on the oracle-made sinogram; converged only "
                           "with a tight f* record and an oracle gap <= tol")


def run_ours(args, ws, rank, local):
    import torch
    import paper_1810_13100_gb300 as ncs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import synth
    W = synth.WORKLOADS[WORKLOAD]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    n, m = N * N, na * nd
    plan = ncs.Plan(N, na, nd, W["lam"], NCS_PARAMS["alpha"], beta=NCS_PARAMS["beta"], gamma=NCS_PARAMS["gamma"],
                    tv=W["tv"], check_every=CHECK_EVERY, h_probes=NCS_PARAMS["h_probes"], fwd_kernel=args.fwd_kernel)
    W, pr = make_inputs(args.seed + rank, gpu_projector(plan, dev))
    b = torch.from_numpy(pr["b"].ravel()).to(dev)
    x = torch.zeros(n, device=dev)
    u = torch.zeros(m, device=dev)
    v = torch.zeros(2 * n, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = plan.stream
    cur = torch.cuda.current_stream()

    def one_step(k):
        plan.step(x, u, v, None, b, n_iter=1)
        if (k + 1) % CHECK_EVERY == 0:
            plan.objective(x, b)                  # FP64 reduction read by the host

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    # the dominant kernel class, from an untimed pass with every kernel bracketed; inside the
    # timed region only it carries events
    plan.profile(True)
    for k in range(CHECK_EVERY):
        one_step(k)
    torch.cuda.synchronize()
    pre = plan.profile_read()
    plan.profile(False)
    dom_name = max(pre.items(), key=lambda kv: kv[1][0])[0]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    plan.profile_mask([dom_name])
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.fill_(float(k))                         # evict L2 (untimed)
            stream.wait_stream(cur)
            starts[k].record(stream)
            one_step(k)
            ends[k].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(ws)
    kern_timed = plan.profile_read()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = sum(step_ms)
    t_max = reduce_max(t_ms, ws)
    total_iters = reduce_sum(args.steps, ws)
    value = total_iters / (t_max / 1000.0)
    # the same steps again (untimed) with every kernel class bracketed: shares and launches
    plan.profile(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        stream.wait_stream(cur)
        one_step(k)
    torch.cuda.synchronize()
    kern = plan.profile_read()
    plan.profile(False)
    launches = sum(plan.kernel_launches.values())

    # ---- roofline of the dominant kernel (algorithmic work / its duration in the timed region)
    peaks, peak_kind = load_peaks()
    dom_ms, dom_n = kern_timed[dom_name] if kern_timed.get(dom_name, (0, 0))[1] else kern[dom_name]
    clk_sum = clk.summary()
    nnz = plan.nnz()
    roof = projector_roofline(dom_name, dom_ms / dom_n, nnz, peaks, dev, load_counters(WORKLOAD))
    # whole-iteration algorithmic bytes (FP32 state read + written once, b read, spectrum round trips)
    it_bytes = 4.0 * (10 * n + 3 * m)
    it_gbs = it_bytes / (t_ms / args.steps / 1000.0) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)

    # ---- end to end through the Python API with host buffers
    e2e = None
    if not args.skip_e2e:
        b_host = torch.from_numpy(pr["b"].ravel()).pin_memory()
        x_host = torch.empty(n, dtype=torch.float32).pin_memory()
        xe = torch.zeros(n, device=dev)
        ue = torch.zeros(m, device=dev)
        ve = torch.zeros(2 * n, device=dev)
        be = torch.empty(m, device=dev)
        k_e2e = max(10, min(args.steps, 200))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(k_e2e):
            be.copy_(b_host, non_blocking=True)
            plan.step(xe, ue, ve, None, be, n_iter=1)
            if (k + 1) % CHECK_EVERY == 0:
                plan.objective(xe, be)
            x_host.copy_(xe, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": reduce_sum(k_e2e, ws) / reduce_max(dt, ws), "unit": "it/s",
               "h2d_bytes_per_step": 4 * m, "d2h_bytes_per_step": 4 * n}

    # ---- time to 1e-4 gap, NCS vs PDHG vs ADMM (same GPU, same inputs, zero start), on every
    # seed of the workload that has the oracle's f* (this rank's seed first); each solver's
    # setup (plan tables, M and its (A3) power iteration for NCS, lambda_max(A^T A) for PDHG)
    # is timed too, and every stopping point is kept for the oracle's own check (CPU leg)
    ttg = None
    stops = {}
    if not args.skip_ttg:
        ttg, stops = time_to_gap(args, rank, ncs, plan, W, N, na, nd, dev)
    # ---- cuFFT as a timing reference for the hand-written FFT solve (A2, A3)
    fft_ref = None
    if rank == 0:
        fft_ref = cufft_reference(N, dev)
        ours = [kern[k] for k in ("fft_rows_fwd", "fft_cols_solve", "fft_rows_inv") if k in kern and kern[k][1]]
        fft_ref["ours_ms"] = sum(v[0] / v[1] for v in ours) if len(ours) == 3 else None

    # ---- algorithmic bytes of the streaming kernels (FP32 state read / written once) and the
    # projector pair's taps per second, from their event-timed durations
    hs = 8 * (N // 2 + 1) * N                       # half spectrum, complex64
    pair = 8 * N * (N + 8)                          # one pair image
    stream_bytes = {"fft_rows_fwd": 4 * n + hs, "fft_cols_solve": 2 * hs + hs // 2,
                    "fft_rows_inv": hs + 12 * n, "tv_prox_transpose": 20 * n + 2 * pair}
    bandwidth = {}
    for k, nb in stream_bytes.items():
        if k in kern and kern[k][1]:
            t = kern[k][0] / kern[k][1] / 1000.0
            bandwidth[k] = {"bytes_per_launch": nb, "gbs": nb / t / 1e9, "frac_of_hbm": nb / t / 1e9 / hbm}
    taps = {k: nnz / (kern[k][0] / kern[k][1] / 1000.0) for k in ("joseph_gather", "joseph_fwd")
            if k in kern and kern[k][1]}

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        r = oracle_rate(args.seed, budget_s=args.cpu_seconds)
        cpu = {"value": r["rate"], "unit": "it/s", "cores": r["cores"], "kind": "oracle",
               "sample": "%d FP64 oracle NCS iterations of the 512x512 workload from zero (%.1f s)"
                         % (r["iters"], r["seconds"])}
        one = oracle_rate_one_core(args.seed, budget_s=max(3.0, args.cpu_seconds / 3))
        if one:
            cpu["one_core"] = {"value": one["rate"], "unit": "it/s", "cores": 1,
                               "sample": "%d FP64 oracle NCS iterations, OMP_NUM_THREADS=1 (%.1f s)"
                                         % (one["iters"], one["seconds"])}
        if ttg and ttg.get("ncs_median_iters"):
            cpu["time_to_gap_s_estimate"] = ttg["ncs_median_iters"] / r["rate"]
            cpu["time_to_gap_estimate_kind"] = "the GPU's iterations to the 1e-4 gap / the oracle's iterations per second"
        if ttg:
            oracle_check_stops(ttg, stops)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "512x512 TV-CT, 720 angles x 730 bins, iso TV lambda 0.005, 20 ellipses, "
                                   "0.5%% noise, seed %d" % args.seed,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed before every timed step (256 MiB write, untimed)",
                       "check_every": CHECK_EVERY, "ncs": NCS_PARAMS,
                       "fwd_kernel": "strips of %d rows (%d)" % (plan.fwd_strips()[1], plan.fwd_strips()[0])
                       if plan.fwd_strips()[0] else "row walk"},
            "roofline": roof,
            "iteration_hbm": {"achieved": it_gbs, "peak": hbm, "unit": "GB/s", "frac": it_gbs / hbm,
                              "algorithmic_bytes_per_iter": it_bytes, "peak_kind": peak_kind},
            "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in kern.items()},
            "kernel_share": {k: v[0] / max(1e-12, sum(w[0] for w in kern.values())) for k, v in kern.items()},
            "gpu_launches": launches,
            "e2e": e2e, "time_to_gap": ttg, "cpu_baseline": cpu, "clocks": clk_sum, "fft_reference": fft_ref,
            "streaming_kernels": bandwidth, "projector_taps_per_s": taps,
        }
        print(json.dumps(line), flush=True)
    plan.close()


def run_batch(args, ws, rank, local):
    """64 independent TV-CT slices of uneven sizes (sides drawn by seed from
    {256, 384, 512}, round(1.4 side) angles, side + 2 bins, the 512x512 workload's
    phantom and noise model) solved together by ncs_batch_solve.  Prints one JSON
    line: slice-iterations per second over K iterations of every slice, per
    precision variant."""
    import torch
    import paper_1810_13100_gb300 as ncs
    import synth
    torch.cuda.set_device(local)
    sides = synth.batch_sides(args.seed, args.slices)
    W = synth.WORKLOADS[WORKLOAD]
    out = {}
    for prec in ("fp32", "bf16"):
        plans, bs, xs = [], [], []
        for i, N in enumerate(sides):
            na, nd = int(round(1.4 * N)), N + 2
            plans.append(ncs.Plan(N, na, nd, W["lam"], NCS_PARAMS["alpha"], beta=NCS_PARAMS["beta"], tv=W["tv"],
                                  precision=prec, autotune=True, check_every=CHECK_EVERY))
            pr = synth.ct_problem(1000 * args.seed + i, N, na, nd, W["n_ellipses"], W["noise_frac"],
                                  gpu_projector(plans[-1], "cuda"))
            bs.append(torch.from_numpy(pr["b"].ravel()).cuda())
            xs.append(torch.zeros(N * N, device="cuda"))
        batch = ncs.Batch(plans)
        lanes = batch.tune_lanes(bs, xs, iters=max(args.warmup, 10))     # untimed setup
        batch.solve(bs, xs, tol=0.0, max_iter=max(args.warmup, 10), f_stars=[-1e300] * len(plans))
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(local) as clk:
            code, reps = batch.solve(bs, xs, tol=0.0, max_iter=args.steps, f_stars=[-1e300] * len(plans))
        barrier(ws)
        ms = reps[0]["time_ms"]
        t_max = reduce_max(ms, ws)
        total = reduce_sum(args.steps * len(plans), ws)
        # kernels per iteration of each slice, counted by its plan's profiler on one untimed
        # step; a solve adds the TV sum and the FP64 finalisation every check_every iterations
        kpi = []
        for p_, b_, x_ in zip(plans, bs, xs):
            m_ = p_.m
            u_ = torch.zeros(m_, device="cuda", dtype=torch.bfloat16 if prec == "bf16" else torch.float32)
            v_ = torch.zeros(2 * p_.n, device="cuda", dtype=u_.dtype)
            xt_ = torch.zeros(p_.n, device="cuda")
            p_.profile(True)
            p_.step(xt_, u_, v_, None, b_, n_iter=1)
            p_.profile_read()
            p_.profile(False)
            kpi.append(sum(p_.kernel_launches.values()))
        launches = sum(args.steps * k + 2 * (args.steps // CHECK_EVERY) for k in kpi)
        # the same slices one after another, each by its own solve on its plan's stream
        seq_ms = None
        if prec == "fp32":
            for x in xs:
                x.zero_()
            torch.cuda.synchronize()
            seq_ms = 0.0
            for p_, b_, x_ in zip(plans, bs, xs):
                rep_ = p_.solve(b_, x_, tol=0.0, max_iter=args.steps, f_star=-1e300)
                seq_ms += rep_["time_ms"]
        pix = reduce_sum(args.steps * sum(N * N for N in sides), ws)
        # algorithmic HBM bytes of one iteration of every slice (FP32 state read + written
        # once, b read, spectrum round trips: 4 (10 n + 3 m) per slice; BF16 storage halves
        # the dual streams, which is not credited here)
        it_bytes = sum(4.0 * (10 * Ns * Ns + 3 * int(round(1.4 * Ns)) * (Ns + 2)) for Ns in sides)
        gbs = it_bytes / (t_max / args.steps / 1000.0) / 1e9
        peaks, peak_kind = load_peaks()
        out[prec] = {"slice_iters_per_s": total / (t_max / 1000.0), "pixel_iters_per_s": pix / (t_max / 1000.0),
                     "hbm": {"algorithmic_bytes_per_batch_iteration": it_bytes, "achieved_gbs": gbs,
                             "peak_gbs": peaks.get("hbm_gbs", 6800.0), "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                             "peak_kind": peak_kind},
                     "ms_per_batch_iteration": t_max / args.steps, "clocks": clk.summary(), "lanes": lanes,
                     "gather_parts": [p.info()["gather_parts"] for p in plans[:4]], "gpu_launches": launches}
        if seq_ms is not None:
            out[prec]["sequential"] = {"slice_iters_per_s": args.steps * len(plans) / (seq_ms / 1000.0),
                                       "ms": seq_ms, "what": "the same slices and iterations, one plan's "
                                       "ncs_solve after another (CUDA graphs of check_every iterations each)"}
            out[prec]["speedup_vs_sequential"] = seq_ms / ms
        batch.close()
        for p in plans:
            p.close()
    if rank == 0:
        line = {"metric": "batched NCS slice-iterations/s (64 uneven TV-CT slices)", "value":
                out["fp32"]["slice_iters_per_s"], "unit": "slice-it/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": out["fp32"]["ms_per_batch_iteration"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "%d slices, sides %s, round(1.4 side) angles, side + 2 bins, iso TV "
                                       "lambda 0.005, seed %d" % (len(sides), sorted(set(sides)), args.seed),
                           "sides": sides, "l2": "working set exceeds L2 (not flushed)"},
                "gpu_launches": out["fp32"]["gpu_launches"], "variants": out}
        print(json.dumps(line), flush=True)


PET_NCS = dict(alpha=1.0, beta=1.0)      # {1,3} x 10^p grid (Sec. 5)
PET_PDHG = dict(alpha=0.1, beta=0.3)


def run_pet(args, ws, rank, local):
    """The 256x256 TV-PET workload (180 angles, 257 bins, 15-ellipse activity, 1e6 counts,
    10% uniform background, KL data term, anisotropic TV lambda 0.02, nonnegativity): NCS
    iterations/s, and NCS and PDHG from zero to the 1e-4 relative gap against the oracle's f*."""
    import numpy as np
    import torch
    import paper_1810_13100_gb300 as ncs
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = synth.WORKLOADS["pet256"]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    seed = args.seed + rank
    plan = ncs.Plan(N, na, nd, W["lam"], PET_NCS["alpha"], beta=PET_NCS["beta"], data="kl", tv=W["tv"],
                    nonneg=True, check_every=CHECK_EVERY)
    pr = synth.pet_problem(seed, N, na, nd, W["n_ellipses"], gpu_projector(plan, dev))
    b = torch.from_numpy(pr["b"].ravel()).to(dev)
    bg = torch.from_numpy(pr["r_bg"].ravel()).to(dev)
    n, m = N * N, na * nd
    x = torch.zeros(n, device=dev); u = torch.zeros(m, device=dev)
    v = torch.zeros(2 * n, device=dev); sv = torch.zeros(n, device=dev)
    plan.step(x, u, v, sv, b, bg, n_iter=max(args.warmup, 3))
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(plan.stream)
        plan.step(x, u, v, sv, b, bg, n_iter=args.steps)
        e1.record(plan.stream)
        torch.cuda.synchronize()
    barrier(ws)
    t_max = reduce_max(e0.elapsed_time(e1), ws)
    rate = reduce_sum(args.steps, ws) / (t_max / 1000.0)
    # the same steps again (untimed), every kernel class bracketed: the kernels they launch
    plan.profile(True)
    plan.step(x, u, v, sv, b, bg, n_iter=args.steps)
    plan.profile_read()
    plan.profile(False)
    launches = sum(plan.kernel_launches.values())
    ttg = None
    gold = load_golden("pet256", seed)
    if gold and not args.skip_ttg:
        fs = gold["f_star"]
        ttg = {"tol": TTG_TOL, "gpu_stop_tol": TTG_STOP, "f_star": fs, "oracle_iters": gold.get("iterations"),
               "f_star_tight": bool(gold.get("tight", False))}
        stops = {}
        if "b_sum" in gold:
            bd = b.double()
            ttg["b_rel_diff"] = {"sum": abs(bd.sum().item() - gold["b_sum"]) / abs(gold["b_sum"]),
                                 "sumsq": abs((bd * bd).sum().item() - gold["b_sumsq"]) / gold["b_sumsq"]}
        xs = torch.zeros(n, device=dev)
        rep = plan.solve(b, xs, tol=TTG_STOP, max_iter=20000, f_star=fs, bg=bg)
        ttg["ncs"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        stops["ncs"] = xs.double().cpu().numpy()
        pplan = ncs.Plan(N, na, nd, W["lam"], PET_PDHG["alpha"], beta=PET_PDHG["beta"], data="kl", tv=W["tv"],
                         nonneg=True, check_every=CHECK_EVERY)
        xs.zero_()
        rep = pplan.pdhg_solve(b, xs, tol=TTG_STOP, max_iter=60000, f_star=fs, bg=bg)
        ttg["pdhg"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        stops["pdhg"] = xs.double().cpu().numpy()
        pplan.close()
        if rank == 0 and not args.skip_cpu:
            oracle_check_one(ttg, "pet256", seed, stops)
    plan.close()
    if rank == 0:
        line = {"metric": "TV-PET NCS iterations/s and time to the 1e-4 gap vs PDHG (256x256)", "value": rate,
                "unit": "it/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "256x256 TV-PET, 180 angles x 257 bins, 15 ellipses, 1e6 counts, 10%% "
                                       "background, KL + aniso TV lambda 0.02 + nonnegativity, seed %d" % seed,
                           "ncs": PET_NCS, "pdhg": PET_PDHG, "l2": "resident (not flushed)"},
                "gpu_launches": launches, "time_to_gap": ttg, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


FAN_NCS = dict(alpha=0.01, beta=0.01, h_probes=128)   # {1,3} x 10^p grid on this workload (seed 0)
FAN_PDHG = dict(alpha=0.001, beta=0.001)
FAN_ADMM = dict(alpha=0.1, beta=0.1, n_cg=10)          # the 512x512 parallel beam's ADMM point


def fan_plan(ncs, W, params, **kw):
    import synth
    return ncs.Plan(W["N"], W["n_angles"], W["n_det"], W["lam"], params["alpha"], beta=params["beta"], tv=W["tv"],
                    src_dist=W["src_dist"], fan_pitch=synth.fan_pitch(W["N"], W["src_dist"], W["n_det"], W["cover"]),
                    check_every=CHECK_EVERY, **kw)


def run_fan(args, ws, rank, local):
    """The 512x512 fan-beam TV-CT workload (Sec. 4, fan beam geometry; 720 source positions on
    a full turn at 1024 pixels from the centre, 768 equiangular channels spanning the image's
    circle, 20 ellipses, 0.5% noise, isotropic TV lambda 0.005): NCS iterations/s with M from
    eq. (H-fan), L2 flushed before each step, the FP64 objective every 10 steps; per-kernel
    shares; the roofline of the dominant kernel; NCS and PDHG from zero to the 1e-4 gap against
    the oracle's f* when it is stored."""
    import torch
    import paper_1810_13100_gb300 as ncs
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = synth.WORKLOADS["fan512"]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    n, m = N * N, na * nd
    seed = args.seed + rank
    plan = fan_plan(ncs, W, FAN_NCS, h_probes=FAN_NCS["h_probes"], fan_gather=args.fan_gather)
    pr = synth.ct_problem(seed, N, na, nd, W["n_ellipses"], W["noise_frac"], gpu_projector(plan, dev))
    b = torch.from_numpy(pr["b"].ravel()).to(dev)
    x = torch.zeros(n, device=dev); u = torch.zeros(m, device=dev); v = torch.zeros(2 * n, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream, cur = plan.stream, torch.cuda.current_stream()

    def one_step(k):
        plan.step(x, u, v, None, b, n_iter=1)
        if (k + 1) % CHECK_EVERY == 0:
            plan.objective(x, b)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    plan.profile_mask(["joseph_gather"])
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.fill_(float(k))
            stream.wait_stream(cur)
            starts[k].record(stream)
            one_step(k)
            ends[k].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(ws)
    kern_timed = plan.profile_read()
    t_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    t_max = reduce_max(t_ms, ws)
    value = reduce_sum(args.steps, ws) / (t_max / 1000.0)
    plan.profile(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        stream.wait_stream(cur)
        one_step(k)
    torch.cuda.synchronize()
    kern = plan.profile_read()
    plan.profile(False)
    launches = sum(plan.kernel_launches.values())
    peaks, peak_kind = load_peaks()
    dom_name = max(kern.items(), key=lambda kv: kv[1][0])[0]
    dom_ms, dom_n = kern_timed[dom_name] if kern_timed.get(dom_name, (0, 0))[1] else kern[dom_name]
    nnz = plan.nnz()
    ncu_name = None
    if dom_name == "joseph_gather":
        ncu_name = "k_gather_fan" if args.fan_gather == "quads" else "k_gather_fan_lines"
    roof = projector_roofline(dom_name, dom_ms / dom_n, nnz, peaks, dev, load_counters("fan512"), ncu_name)
    tot_ms = sum(t for t, _ in kern.values())
    kernels = {k: {"ms_per_launch": t / c if c else None, "launches": c, "share": t / tot_ms if tot_ms else None}
               for k, (t, c) in kern.items()}
    ttg = None
    gold = load_golden("fan512", seed)
    if gold and not args.skip_ttg:
        fs = gold["f_star"]
        bd = b.double()
        ttg = {"tol": TTG_TOL, "gpu_stop_tol": TTG_STOP, "f_star": fs, "oracle_iters": gold.get("iterations"),
               "f_star_tight": bool(gold.get("tight", False)),
               "f_star_decrease_last_1000_rel": gold["decrease_last_1000"] / abs(fs),
               "b_rel_diff": {"sum": abs(bd.sum().item() - gold["b_sum"]) / abs(gold["b_sum"]),
                              "sumsq": abs((bd * bd).sum().item() - gold["b_sumsq"]) / gold["b_sumsq"]}}
        stops = {}
        xs = torch.zeros(n, device=dev)
        rep = plan.solve(b, xs, tol=TTG_STOP, max_iter=4000, f_star=fs)
        ttg["ncs"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        stops["ncs"] = xs.double().cpu().numpy()
        # PDHG's step comes from lambda_max(A^T A) by the plan's full power iteration
        pplan = fan_plan(ncs, W, FAN_PDHG, h_probes=1, fan_gather=args.fan_gather)
        xs.zero_()
        rep = pplan.pdhg_solve(b, xs, tol=TTG_STOP, max_iter=args.pdhg_extended, f_star=fs)
        ttg["pdhg"] = {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}
        stops["pdhg"] = xs.double().cpu().numpy()
        pplan.close()
        aplan = fan_plan(ncs, W, FAN_ADMM, h_probes=FAN_NCS["h_probes"], fan_gather=args.fan_gather)
        xs.zero_()
        rep = aplan.admm_solve(b, xs, tol=TTG_STOP, max_outer=ADMM_CAP, n_cg=FAN_ADMM["n_cg"], f_star=fs)
        ttg["admm"] = dict(FAN_ADMM, outer=rep["iters"], time_ms=rep["time_ms"], gap=rep["gap"],
                           status=rep["status"])
        stops["admm"] = xs.double().cpu().numpy()
        aplan.close()
        if rank == 0 and not args.skip_cpu:
            oracle_check_one(ttg, "fan512", seed, stops)
    plan.close()
    if rank == 0:
        line = {"metric": "fan-beam TV-CT NCS iterations/s (512x512, 720 views x 768 channels)", "value": value,
                "unit": "it/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "512x512 fan-beam TV-CT, 720 views on [0, 2pi), 768 equiangular channels, "
                                       "source at 1024 px, 20 ellipses, 0.5%% noise, iso TV lambda 0.005, seed %d"
                                       % seed, "ncs": FAN_NCS, "pdhg": FAN_PDHG, "admm": FAN_ADMM,
                           "fan_gather": args.fan_gather,
                           "l2": "flushed before every step (256 MiB write, untimed)"},
                "roofline": roof, "kernels": kernels, "gpu_launches": launches, "peaks": peak_kind,
                "time_to_gap": ttg, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


CONE_NCS = dict(alpha=0.003, beta=0.003, h_probes=128)  # {1,3} x 10^p grid: fastest to the gap on cone128


def run_cone(args, ws, rank, local):
    """A cone-beam TV-CT workload (Sec. 4, cone beam geometry): cone128, a 128 x 128 x 32 volume,
    180 source positions on a full turn at 256 voxels from the centre, 32 detector rows x 192
    equiangular channels, 12 ellipsoids; or cone64, the same proportions at half the size; 0.5%
    noise, isotropic TV lambda 0.005.  3-D NCS iterations/s (L2 flushed before each step, the
    FP64 objective every 10 steps), and NCS from zero to the 1e-4 gap against the oracle's stored
    minimum (reported without a convergence claim while that record is not tight)."""
    import numpy as np
    import torch
    import paper_1810_13100_gb300 as ncs
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = synth.WORKLOADS[args.workload]
    N, Nz, na, nr, nd, R = W["N"], W["Nz"], W["n_angles"], W["n_rows"], W["n_det"], W["src_dist"]
    pitch = synth.fan_pitch(N, R, nd, W["cover"])
    rp = synth.cone_row_pitch(N, Nz, R, nr, W["cover"])
    seed = args.seed + rank
    t0 = time.perf_counter()
    plan = ncs.ConePlan(N, Nz, na, nr, nd, R, pitch, rp, W["lam"], CONE_NCS["alpha"], beta=CONE_NCS["beta"],
                        tv=W["tv"], h_probes=CONE_NCS["h_probes"], check_every=CHECK_EVERY)
    setup_ms = _sync_ms(t0)
    cone = ncs.Cone(N, Nz, na, nr, nd, R, pitch, rp)

    def project(x):
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32).ravel()).to(dev)
        return cone.apply_K(t).cpu().numpy().astype(np.float64).reshape(na, nr, nd)

    pr = synth.ct3d_problem(seed, N, Nz, na, nr, nd, W["n_ellipses"], W["noise_frac"], project)
    b = torch.from_numpy(pr["b"].ravel()).to(dev)
    n, m = N * N * Nz, na * nr * nd
    x = torch.zeros(n, device=dev); u = torch.zeros(m, device=dev); v = torch.zeros(3 * n, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream, cur = plan.stream, torch.cuda.current_stream()

    def one_step(k):
        plan.step(x, u, v, b, n_iter=1)
        if (k + 1) % CHECK_EVERY == 0:
            plan.objective(x, b)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    k_before = plan.kernels()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.fill_(float(k))
            stream.wait_stream(cur)
            starts[k].record(stream)
            one_step(k)
            ends[k].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(ws)
    launches = plan.kernels() - k_before
    t_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    t_max = reduce_max(t_ms, ws)
    value = reduce_sum(args.steps, ws) / (t_max / 1000.0)
    ttg = None
    gold = load_golden(args.workload, seed)
    if gold and not args.skip_ttg:
        fs = gold["f_star"]
        bd = b.double()
        xs = torch.zeros(n, device=dev)
        rep = plan.solve(b, xs, tol=TTG_STOP, max_iter=4000, f_star=fs)
        ttg = {"tol": TTG_TOL, "gpu_stop_tol": TTG_STOP, "f_star": fs, "oracle_iters": gold.get("iterations"),
               "f_star_tight": bool(gold.get("tight", False)),
               "f_star_decrease_last_1000_rel": gold["decrease_last_1000"] / abs(fs),
               "b_rel_diff": {"sum": abs(bd.sum().item() - gold["b_sum"]) / abs(gold["b_sum"]),
                              "sumsq": abs((bd * bd).sum().item() - gold["b_sumsq"]) / gold["b_sumsq"]},
               "ncs": {k: rep[k] for k in ("iters", "time_ms", "gap", "status")}, "setup_ms": setup_ms}
        ttg["ncs"]["with_setup_ms"] = rep["time_ms"] + setup_ms
        if rank == 0 and not args.skip_cpu:
            # the FP64 oracle's objective at the stop, on the sinogram the stored f* was computed
            # for (made with the oracle's own cone-beam K)
            from oracle import cone as oc
            g = oc.ConeGeometry(N, Nz, na, nr, nd, R, pitch, rp)
            opr = synth.ct3d_problem(seed, N, Nz, na, nr, nd, W["n_ellipses"], W["noise_frac"], lambda z: oc.K(z, g))
            P = oc.Problem(g, opr["b"].astype(np.float64), lam=W["lam"], alpha=1.0, beta=1.0, tv=W["tv"])
            f = oc.objective(P, xs.double().cpu().numpy().reshape(g.shape))
            ttg["ncs"]["oracle_f"] = f
            ttg["ncs"]["oracle_gap"] = (f - fs) / abs(fs)
            ttg["ncs_converged_oracle"] = int(ttg["f_star_tight"] and rep["status"] == 0
                                              and ttg["ncs"]["oracle_gap"] <= TTG_TOL)
        if not ttg["f_star_tight"]:
            ttg["claim"] = "none: the stored reference minimum is not tight (its last 1000 oracle iterations " \
                           "lowered f by more than 1e-7 relative)"
    plan.close()
    cone.close()
    if rank == 0:
        shape = "%dx%dx%d, %d views x %d rows x %d channels" % (N, N, Nz, na, nr, nd)
        line = {"metric": "cone-beam 3-D TV-CT NCS iterations/s (%s)" % shape,
                "value": value, "unit": "it/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "%s cone-beam TV-CT, views on [0, 2pi), source at %g voxels, %d ellipsoids, "
                                       "0.5%% noise, iso TV lambda 0.005, seed %d" % (shape, R, W["n_ellipses"], seed),
                           "ncs": CONE_NCS,
                           "l2": "flushed before every step (256 MiB write, untimed)"},
                "setup_ms": setup_ms, "gpu_launches": launches, "time_to_gap": ttg, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def unet_conv_flops(H, W, levels, base):
    """FLOPs of one forward pass of the U-Net's 3x3 convolutions (2 per multiply-add)."""
    c = [base << l for l in range(levels)]
    f = 0
    for l in range(levels):
        hw = (H >> l) * (W >> l)
        f += 2 * 9 * hw * (1 if l == 0 else c[l - 1]) * c[l] + 2 * 9 * hw * c[l] * c[l]
    for l in range(levels - 1):
        hw = (H >> l) * (W >> l)
        f += 2 * 9 * hw * (c[l + 1] + c[l]) * c[l] + 2 * 9 * hw * c[l] * c[l]
    return f


def run_unet(args, ws, rank, local):
    """Train steps of the warm-start U-Net (4 levels, base 32, 512x512; forward, backward
    and Adam in the library's kernels) on a seeded phantom with noise as input and the
    phantom as target.  One JSON line: train steps/s, with a tensor-core roofline of the
    convolutions (forward + data gradient + weight gradient) against the measured bf16 peak."""
    import numpy as np
    import torch
    import paper_1810_13100_gb300 as ncs
    import synth
    torch.cuda.set_device(local)
    H, levels, base = 512, 4, 32
    x_true, z = synth.ct_phantom(args.seed + rank, H, 1, H * H, 20)
    xin = torch.from_numpy((x_true.ravel() + 0.05 * z.ravel()).astype(np.float32)).cuda()
    tgt = torch.from_numpy(x_true.ravel()).cuda()
    net = ncs.UNet(H, H, levels=levels, base=base, seed=args.seed)
    for _ in range(max(args.warmup, 3)):
        net.train_step(xin, tgt, 1e-4)
    torch.cuda.synchronize()
    barrier(ws)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            net.train_step(xin, tgt, 1e-4)        # synchronises (reads the loss)
        dt = time.perf_counter() - t0
    barrier(ws)
    t_max = reduce_max(dt, ws)
    steps = reduce_sum(args.steps, ws)
    ff = unet_conv_flops(H, H, levels, base)
    # backward: data gradient of every convolution but the first, and every weight gradient
    first = 2 * 9 * H * H * 1 * base
    flops = ff + (ff - first) + ff
    peaks, kind = load_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    ach = flops / (t_max / args.steps) / 1e12
    t1 = time.perf_counter()
    for _ in range(20):
        net.forward(xin)
    fwd_ms = (time.perf_counter() - t1) / 20 * 1e3
    net.close()
    if rank == 0:
        line = {"metric": "U-Net train steps/s (warm start: 4 levels, base 32, 512x512, bf16 tensor cores)",
                "value": steps / t_max, "unit": "step/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": "U-Net 4 levels / base 32 on a 512x512 seeded phantom, Adam, batch 1"},
                "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                             "traffic": None, "work": "%.4g conv FLOP per train step (forward %.4g)" % (flops, ff),
                             "peak_kind": "%s (bf16 burst)" % kind},
                "forward_ms": fwd_ms, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--skip-ttg", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ttg-extended", type=int, default=8000)
    ap.add_argument("--pdhg-extended", type=int, default=20000,
                    help="PDHG iteration cap on the first seed when it misses the gap within the cap")
    ap.add_argument("--admm-grid", action="store_true",
                    help="time the ADMM comparator over a grid of alpha and n_cg on the first seed")
    ap.add_argument("--workload", default="ct512", choices=["ct512", "batch64", "unet", "pet256", "fan512", "cone128", "cone64"])
    ap.add_argument("--slices", type=int, default=64)
    ap.add_argument("--fan-gather", default="auto", choices=["auto", "lines", "quads"],
                    help="fan-beam K^T kernel (fan512 workload)")
    ap.add_argument("--fwd-kernel", default="auto", choices=["auto", "strips", "rows"],
                    help="parallel-beam K kernel of the ct512 step (the time-to-gap plans take the default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on the host of rank 0 only; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    ws, rank, local = dist_setup()
    if args.workload == "batch64":
        run_batch(args, ws, rank, local)
    elif args.workload == "unet":
        run_unet(args, ws, rank, local)
    elif args.workload == "pet256":
        run_pet(args, ws, rank, local)
    elif args.workload == "fan512":
        run_fan(args, ws, rank, local)
    elif args.workload in ("cone128", "cone64"):
        run_cone(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
