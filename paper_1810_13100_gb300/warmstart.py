"""Learned warm start for NCS (not in the paper).

A U-Net (include/ncs.h, ncs_unet_*) maps the Ram-Lak filtered backprojection of a
sinogram to an initial image x^0; NCS then runs unchanged from x^0 (zero duals by
default), so convergence (Sec. 3) is untouched and plain NCS from zero stays the
fallback.  Training pairs are (FBP(b), x_T) with x_T the plain NCS iterate after T
iterations on the same problem; every step runs in the library's kernels (NCS
through ncs_batch_solve, the network through its tensor-core forward and backward).

Command line (phantoms from the repository's seeded generator `synth`):

    python -m paper_1810_13100_gb300.warmstart train --pairs 2000 --target-iters 1000 \
        --epochs 8 --out weights.npz
    python -m paper_1810_13100_gb300.warmstart eval --weights weights.npz --seeds 5000:5200
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from .binding import Batch, Plan, UNet


# ------------------------------------------------------------------ the warm start
class WarmStart:
    """FBP -> U-Net -> x^0 for the geometry of `plan` (square N x N images)."""

    def __init__(self, plan: Plan, levels: int = 4, base: int = 32, seed: int = 0, params=None):
        self.plan = plan
        self.levels, self.base = int(levels), int(base)
        self.net = UNet(plan.N, plan.N, levels=self.levels, base=self.base, seed=seed)
        if params is not None:
            self.net.set_params(params)

    def fbp(self, b, out=None):
        return self.plan.fbp(b, out)

    def x0(self, b, out=None):
        """x^0 = FBP(b) + net(FBP(b)) as a device float32 tensor of N*N."""
        return self.net.forward(self.plan.fbp(b), out)

    def save(self, path: str, meta: dict | None = None) -> None:
        info = {"levels": self.levels, "base": self.base, "N": self.plan.N,
                "n_angles": self.plan.n_angles, "n_det": self.plan.n_det}
        info.update(meta or {})
        np.savez(path, params=self.net.params(), meta=json.dumps(info))

    @staticmethod
    def load(path: str, plan: Plan) -> "WarmStart":
        z = np.load(path)
        info = json.loads(str(z["meta"]))
        if info["N"] != plan.N:
            raise ValueError("weights are for %dx%d images, the plan is %dx%d" % (info["N"], info["N"], plan.N, plan.N))
        return WarmStart(plan, info["levels"], info["base"], params=z["params"])

    def close(self):
        self.net.close()


# ------------------------------------------------------------------ training pairs
def solve_batch(plans, batch, bs, x0s, tol, max_iter, f_stars=None):
    """Solve len(bs) <= len(plans) slices together; returns the reports."""
    k = len(bs)
    if k == len(plans):
        _, reps = batch.solve(bs, x0s, tol=tol, max_iter=max_iter, f_stars=f_stars)
        return reps
    sub = Batch(plans[:k])
    try:
        _, reps = sub.solve(bs, x0s, tol=tol, max_iter=max_iter, f_stars=f_stars)
    finally:
        sub.close()
    return reps


def make_pairs(plans, sinograms, target_iters: int, log=None):
    """Inputs FBP(b) and targets x_T (T = target_iters plain NCS iterations from zero)
    for an iterable of device sinograms, solved len(plans) at a time."""
    import torch
    batch = Batch(plans)
    ins, outs = [], []
    chunk = []
    t0 = time.time()

    def flush():
        xs = [torch.zeros(plans[0].n, device="cuda") for _ in chunk]
        solve_batch(plans, batch, chunk, xs, 0.0, target_iters)
        for b, x in zip(chunk, xs):
            ins.append(plans[0].fbp(b))
            outs.append(x)
        if log:
            log("pairs %d (%.1fs)" % (len(ins), time.time() - t0))
        chunk.clear()

    for b in sinograms:
        chunk.append(b)
        if len(chunk) == len(plans):
            flush()
    if chunk:
        flush()
    batch.close()
    return ins, outs


def train(ws: WarmStart, inputs, targets, epochs: int, lr: float = 1e-3, lr_min: float = 1e-5,
          val_frac: float = 0.05, seed: int = 0, log=None):
    """Adam on mean((x + net(x) - t)^2), one pair per step, cosine learning rate from
    lr to lr_min; the last val_frac of the pairs are held out.  Returns the history."""
    n = len(inputs)
    n_val = max(1, int(round(val_frac * n))) if n > 1 else 0
    tr = list(range(n - n_val))
    rng = np.random.default_rng(seed)
    total = max(1, epochs * len(tr))
    hist = []
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        rng.shuffle(tr)
        run = 0.0
        for i in tr:
            a = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / total))
            run += ws.net.train_step(inputs[i], targets[i], a)
            step += 1
        val = float(np.mean([ws.net.gradient(inputs[i], targets[i])[0] for i in range(n - n_val, n)])) if n_val else None
        hist.append({"epoch": ep, "train_mse": run / max(1, len(tr)), "val_mse": val, "s": time.time() - t0})
        if log:
            log("epoch %d train %.4e val %s (%.1fs)" % (ep, hist[-1]["train_mse"],
                                                      "%.4e" % val if val is not None else "-", time.time() - t0))
    return hist


# ------------------------------------------------------------------ evaluation
def evaluate(plans, ws: WarmStart | None, sinograms, tol: float = 1e-4, cap: int = 4000, ref_iters: int = 8000,
             log=None):
    """Iterations to a relative objective gap `tol` from zero, FBP and (if ws) the
    learned start, per sinogram.  The reference f is the objective of plain NCS
    from zero after ref_iters iterations.  Returns a list of dicts."""
    import torch
    batch = Batch(plans)
    res = []
    bs_all = list(sinograms)
    k = len(plans)
    for c0 in range(0, len(bs_all), k):
        bs = bs_all[c0:c0 + k]
        zeros = lambda: [torch.zeros(plans[0].n, device="cuda") for _ in bs]
        ref = solve_batch(plans, batch, bs, zeros(), 0.0, ref_iters)
        f_ref = [r["f"] for r in ref]
        starts = {"zero": zeros(), "fbp": [plans[0].fbp(b) for b in bs]}
        if ws is not None:
            starts["learned"] = [ws.x0(b) for b in bs]
        f0 = {name: [plans[0].objective(x, b) for x, b in zip(xs, bs)] for name, xs in starts.items()}
        out, wall = {}, {}
        for name, xs in starts.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out[name] = solve_batch(plans, batch, bs, xs, tol, cap, f_stars=f_ref)
            torch.cuda.synchronize()
            wall[name] = (time.perf_counter() - t0) * 1e3 / len(bs)
        prep = {"zero": 0.0, "fbp": 0.0, "learned": 0.0}
        if ws is not None:
            # the learned start's own cost per slice (FBP + network), timed separately
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for bb in bs:
                ws.x0(bb)
            torch.cuda.synchronize()
            prep["learned"] = (time.perf_counter() - t0) * 1e3 / len(bs)
        for j in range(len(bs)):
            row = {"f_ref": f_ref[j]}
            for name in starts:
                r = out[name][j]
                row[name] = {"iters": r["iters"] if r["status"] == 0 else None, "gap0": (f0[name][j] - f_ref[j]) / f_ref[j],
                             "gap": r["gap"], "batch_ms_per_slice": wall[name] + prep.get(name, 0.0)}
            res.append(row)
        if log:
            log("evaluated %d (%s)" % (len(res), "  ".join(
                "%s %.0f" % (nm, np.mean([r[nm]["iters"] or cap for r in res])) for nm in starts)))
    batch.close()
    return res


def time_single(plan: Plan, ws: WarmStart | None, b, f_ref: float, tol: float = 1e-4, cap: int = 4000):
    """Wall time (CUDA events) to the tolerance for one slice from each start, the
    warm start's FBP and network time included."""
    import torch
    out = {}
    starts = ["zero", "fbp"] + (["learned"] if ws is not None else [])
    for name in starts:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if name == "zero":
            x = torch.zeros(plan.n, device="cuda")
        elif name == "fbp":
            x = plan.fbp(b)
        else:
            x = ws.x0(b)
        e1.record()
        torch.cuda.synchronize()
        prep = e0.elapsed_time(e1)
        r = plan.solve(b, x, tol=tol, max_iter=cap, f_star=f_ref)
        out[name] = {"prep_ms": prep, "solve_ms": r["time_ms"], "iters": r["iters"], "status": r["status"],
                     "total_ms": prep + r["time_ms"]}
    return out


# ------------------------------------------------------------------ command line
def _phantom(args):
    import synth
    return synth.ct_phantom(*args)


def _sinograms(pool, seeds, geo, plan):
    """Device sinograms b = K x_true + noise of the seeded phantoms (synth's recipe),
    projected with the plan's K; the phantoms are drawn in worker processes."""
    import torch
    import synth
    N, na, nd, n_ell, noise = geo
    args = [(s, N, na, nd, n_ell) for s in seeds]
    for x_true, z in (pool.imap(_phantom, args, chunksize=2) if pool else map(_phantom, args)):
        Kx = plan.apply_K(torch.from_numpy(x_true.ravel()).cuda()).cpu().numpy()
        b, _ = synth.ct_data(Kx, z, noise)
        yield torch.from_numpy(b.ravel()).cuda()


def main(argv=None):
    import argparse
    import multiprocessing as mp
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("mode", choices=["train", "eval", "both"])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--angles", type=int, default=720)
    ap.add_argument("--bins", type=int, default=730)
    ap.add_argument("--ellipses", type=int, default=20)
    ap.add_argument("--noise", type=float, default=0.005)
    ap.add_argument("--lam", type=float, default=0.005)
    ap.add_argument("--alpha", type=float, default=0.01)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--pair-seed0", type=int, default=10000)
    ap.add_argument("--target-iters", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--slices", type=int, default=32, help="slices solved together")
    ap.add_argument("--seeds", default="5000:5200")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--cap", type=int, default=4000)
    ap.add_argument("--ref-iters", type=int, default=8000)
    ap.add_argument("--time-slices", type=int, default=8)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--out", default="warmstart_weights.npz")
    ap.add_argument("--report", default=None)
    ap.add_argument("--workers", type=int, default=8)
    a = ap.parse_args(argv)
    pool = mp.get_context("spawn").Pool(a.workers) if a.workers > 0 else None   # before any CUDA call
    import torch
    t_start = time.time()

    def log(msg):
        print("[%7.1fs] %s" % (time.time() - t_start, msg), flush=True)

    geo = (a.N, a.angles, a.bins, a.ellipses, a.noise)
    plans = [Plan(a.N, a.angles, a.bins, a.lam, a.alpha, beta=a.alpha, tv="iso") for _ in range(a.slices)]
    log("plans ready (rho %.3f)" % plans[0].power_bound()[1])
    report = {"geometry": {"N": a.N, "angles": a.angles, "bins": a.bins, "ellipses": a.ellipses, "noise": a.noise,
                           "lam": a.lam, "alpha": a.alpha, "beta": a.alpha, "tv": "iso"}}
    ws = None
    if a.mode in ("train", "both"):
        seeds = range(a.pair_seed0, a.pair_seed0 + a.pairs)
        t0 = time.time()
        ins, outs = make_pairs(plans, _sinograms(pool, seeds, geo, plans[0]), a.target_iters, log=log)
        t_pairs = time.time() - t0
        ws = WarmStart(plans[0], a.levels, a.base, seed=1)
        t0 = time.time()
        hist = train(ws, ins, outs, a.epochs, lr=a.lr, log=log)
        t_train = time.time() - t0
        ws.save(a.out, {"pairs": a.pairs, "target_iters": a.target_iters, "epochs": a.epochs, "lr": a.lr})
        report["train"] = {"pairs": a.pairs, "pair_seeds": [a.pair_seed0, a.pair_seed0 + a.pairs],
                           "target_iters": a.target_iters, "epochs": a.epochs, "levels": a.levels, "base": a.base,
                           "n_params": ws.net.n_params, "pairs_s": t_pairs, "train_s": t_train,
                           "steps_per_s": a.epochs * len(ins) / max(t_train, 1e-9), "history": hist}
        del ins, outs
    if a.mode in ("eval", "both"):
        if ws is None and a.weights:
            ws = WarmStart.load(a.weights, plans[0])
        lo, hi = (int(v) for v in a.seeds.split(":"))
        res = evaluate(plans, ws, _sinograms(pool, range(lo, hi), geo, plans[0]), tol=a.tol, cap=a.cap,
                       ref_iters=a.ref_iters, log=log)
        names = [k for k in res[0] if k != "f_ref"]
        summ = {}
        for nm in names:
            its = [r[nm]["iters"] for r in res]
            ok = [i for i in its if i is not None]
            summ[nm] = {"converged": len(ok), "of": len(its), "mean_iters": float(np.mean(ok)) if ok else None,
                        "median_iters": float(np.median(ok)) if ok else None,
                        "mean_gap0": float(np.mean([r[nm]["gap0"] for r in res])),
                        "batch_ms_per_slice": float(np.mean([r[nm]["batch_ms_per_slice"] for r in res]))}
        if "learned" in names:
            pair = [(r["zero"]["iters"], r["learned"]["iters"]) for r in res
                    if r["zero"]["iters"] and r["learned"]["iters"]]
            summ["learned_over_zero_iters"] = float(np.mean([l / z for z, l in pair])) if pair else None
            summ["learned_fewer_than_fbp"] = int(sum(1 for r in res if r["learned"]["iters"] and r["fbp"]["iters"]
                                                    and r["learned"]["iters"] < r["fbp"]["iters"]))
            # per-seed spread of the learned start against FBP (iterations are counted in steps of
            # the solves' check interval)
            d = np.array([r["learned"]["iters"] - r["fbp"]["iters"] for r in res
                          if r["learned"]["iters"] and r["fbp"]["iters"]], dtype=np.float64)
            if len(d) > 1:
                se = float(d.std(ddof=1) / np.sqrt(len(d)))
                summ["learned_minus_fbp_iters"] = {
                    "n": int(len(d)), "mean": float(d.mean()), "std": float(d.std(ddof=1)), "stderr": se,
                    "t": float(d.mean() / se) if se > 0 else None, "fewer": int((d < 0).sum()),
                    "equal": int((d == 0).sum()), "more": int((d > 0).sum()),
                    "relative_mean": float(np.mean([(r["learned"]["iters"] - r["fbp"]["iters"]) / r["fbp"]["iters"]
                                                    for r in res if r["learned"]["iters"] and r["fbp"]["iters"]]))}
        # single-slice wall time on the first few seeds
        tim = []
        bs = list(_sinograms(None, range(lo, lo + a.time_slices), geo, plans[0]))
        for b, r in zip(bs, res):
            tim.append(time_single(plans[0], ws, b, r["f_ref"], tol=a.tol, cap=a.cap))
        for nm in tim[0]:
            summ.setdefault(nm, {})["single_mean_total_ms"] = float(np.mean([t[nm]["total_ms"] for t in tim]))
            summ[nm]["single_mean_prep_ms"] = float(np.mean([t[nm]["prep_ms"] for t in tim]))
        report["eval"] = {"seeds": [lo, hi], "tol": a.tol, "cap": a.cap, "ref_iters": a.ref_iters,
                          "summary": summ, "per_seed": res, "single": tim}
        log("summary " + json.dumps(summ))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)
    if pool:
        pool.close()
    for p in plans:
        p.close()


if __name__ == "__main__":
    main()
