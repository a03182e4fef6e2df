"""Learned initial guess for the Newton-Krylov base-flow solve.

The Newton-Krylov fixed-point method (Sec. 3.1.2, Eq. 43) needs fewer
iterations the closer its start is to the steady state.  The paper starts
from a flow field at hand; here a U-Net (the library's `unet_*` calls)
predicts the base-flow vorticity from the flow parameters, and Newton starts
from that prediction.

Pipeline (all GPU work in the library; this module draws the seeded inputs,
moves tensors and keeps the books):
  1. training labels: base flows for seeded (Re, D) pairs by Newton, in
     order of Re, each started from the previous converged flow (parameter
     continuation; the first, and any continuation that fails, from the
     plain start).  The Re-sorted pairs are cut into `chains` contiguous
     runs: the first pair of each run is solved in sequence (each from the
     previous run's first flow), then the runs continue concurrently, one
     host thread and CUDA stream each -- a small grid leaves the GPU idle
     between the launches of one solve, which other solves fill;
  2. train the network on (features, label) pairs with Adam;
  3. for held-out (Re, D): Newton from the network's prediction against
     Newton from the plain start -- selective frequency damping (Sec. 3.1.1,
     Eq. 40) from rest for a fixed number of steps -- in iterations,
     Jacobian products and seconds.

Run as ``python -m paper_1804_03859_gb300.learned_guess [options]``; prints
one JSON line (two with --c4).
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time

import numpy as np

from . import nsstab

FEATURES = 3


def features(nx: int, ny: int, Re: float, D: float, Lx: float = 16.0, Ly: float = 8.0,
             cyl_x: float = 4.0, cyl_y: float = 4.0) -> np.ndarray:
    """Network input [3][ny][nx]: a Gaussian bump of radius D/2 at the
    cylinder (periodic distance), the Reynolds number and the diameter as
    constant planes, each scaled to order one."""
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    ddx = (x - cyl_x + 0.5 * Lx) % Lx - 0.5 * Lx
    ddy = (y - cyl_y + 0.5 * Ly) % Ly - 0.5 * Ly
    r2 = ddx[None, :] ** 2 + ddy[:, None] ** 2
    bump = np.exp(-r2 / (0.5 * D) ** 2)
    return np.stack([bump, np.full((ny, nx), (Re - 95.0) / 55.0), np.full((ny, nx), (D - 1.0) / 0.2)])


def he_init(in_ch: int, width: int, seed: int) -> np.ndarray:
    """Seeded initial parameters in the library's flat layout: weights
    normal with variance 2 / fan-in, biases zero."""
    rng = np.random.default_rng(seed)
    c = [width << l for l in range(4)]
    shapes = []
    ci = in_ch
    for l in range(4):
        shapes += [(c[l], ci, 9), (c[l], c[l], 9)]
        ci = c[l]
    for l in (2, 1, 0):
        shapes += [(c[l], c[l + 1] + c[l], 9), (c[l], c[l], 9)]
    shapes.append((1, c[0], 1))
    out = []
    for co, cin, k in shapes:
        out.append(rng.standard_normal(co * cin * k) * math.sqrt(2.0 / (cin * k)))
        out.append(np.zeros(co))
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == nsstab.load_library().unet_param_count(in_ch, width)
    return theta


def train_step_flops(in_ch: int, width: int, ny: int, nx: int, batch: int) -> int:
    """Multiply-add flops of one training step: every 3x3 convolution's
    forward, input-gradient and weight-gradient products (2 P Ci Co 9 each;
    the first layer's input gradient is not formed) and the output layer's
    three products."""
    c = [width << l for l in range(4)]
    convs = []          # (level, ci, co)
    ci = in_ch
    for l in range(4):
        convs += [(l, ci, c[l]), (l, c[l], c[l])]
        ci = c[l]
    for l in (2, 1, 0):
        convs += [(l, c[l + 1] + c[l], c[l]), (l, c[l], c[l])]
    total = 0
    for k, (l, cin, co) in enumerate(convs):
        P = batch * (ny >> l) * (nx >> l)
        total += 2 * P * cin * co * 9 * (2 if k == 0 else 3)
    return total + 3 * 2 * batch * ny * nx * c[0]


def _sync():
    import torch

    torch.cuda.current_stream().synchronize()   # this thread's stream only (chains run concurrently)


def _solve(st, q, args):
    _sync()
    t0 = time.perf_counter()
    rc, r, it, mv = st.newton_krylov_fixedpoint(q, T=args.T, gmres_m=args.gmres_m, tol=args.tol,
                                                max_newton=args.max_newton)
    _sync()
    return {"ok": rc == nsstab.OK, "residual": r, "iters": it, "matvecs": mv, "seconds": time.perf_counter() - t0}


def plain_start(st, args):
    """SFD from rest for args.sfd_steps steps (the start without a model)."""
    import torch

    q = torch.zeros(args.ny, args.nx, dtype=torch.float64, device="cuda")
    _sync()
    t0 = time.perf_counter()
    st.sfd_baseflow(q, chi=args.chi, Delta=args.Delta, tol=0.0, max_steps=args.sfd_steps,
                    check_every=args.sfd_steps)
    _sync()
    return q, time.perf_counter() - t0


def sample_params(n: int, seed: int, re_min: float = 40.0, re_max: float = 150.0):
    rng = np.random.default_rng(seed)
    return [(float(rng.uniform(re_min, re_max)), float(rng.uniform(0.8, 1.2))) for _ in range(n)]


def run(args, keep: dict | None = None) -> dict:
    """The experiment; `keep` (optional) receives the trained network
    ("net") and the label scale ("scale") for a later solve."""
    import torch

    dt = args.dt if args.dt > 0 else 0.01 * 128 / args.nx
    kw = dict(nx=args.nx, ny=args.ny, dt=dt)
    t_all = time.perf_counter()

    # 1. dataset: training labels by continuation in Re, test pairs from the plain start
    def from_plain(Re, D):
        st = nsstab.Stepper(Re=Re, cyl_D=D, **kw)
        q, t_sfd = plain_start(st, args)
        rec = _solve(st, q, args)
        rec.update(Re=Re, D=D, sfd_seconds=t_sfd, label=q.clone())
        return rec

    def continue_from(prev, Re, D):
        rec = None
        if prev is not None:
            st = nsstab.Stepper(Re=Re, cyl_D=D, **kw)
            q = prev.clone()
            rec = _solve(st, q, args)
            rec.update(Re=Re, D=D, label=q.clone())
            del st
        if rec is None or not rec["ok"]:
            rec = from_plain(Re, D)
        return rec

    t0 = time.perf_counter()
    pairs = sorted(sample_params(args.train, args.seed, args.re_min, args.re_max))
    K = max(1, min(args.chains, len(pairs)))
    runs = [list(c) for c in np.array_split(np.arange(len(pairs)), K) if len(c)]
    # the first pair of every run, in sequence
    heads, prev = [], None
    for r in runs:
        rec = continue_from(prev, *pairs[r[0]])
        heads.append(rec)
        if rec["ok"]:
            prev = rec["label"]
    # the rest of every run, runs concurrently (one thread and stream each)
    results = [[h] for h in heads]
    errors = []

    def chain(k):
        import torch

        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                prev = heads[k]["label"] if heads[k]["ok"] else None
                for i in runs[k][1:]:
                    rec = continue_from(prev, *pairs[i])
                    results[k].append(rec)
                    if rec["ok"]:
                        prev = rec["label"]
                _sync()
        except Exception as e:   # reported below; a thread must not die silently
            errors.append(repr(e))

    threads = [threading.Thread(target=chain, args=(k,)) for k in range(len(runs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise RuntimeError("label generation failed: " + "; ".join(errors))
    train = [rec for chain_recs in results for rec in chain_recs if rec["ok"]]
    t_labels = time.perf_counter() - t0
    test = [from_plain(Re, D) for Re, D in sample_params(args.test, args.seed + 1, args.re_min, args.re_max)]
    t_data = time.perf_counter() - t0
    if not train:
        return {"error": "no training base flow converged"}

    # 2. training
    X = torch.from_numpy(np.stack([features(args.nx, args.ny, r["Re"], r["D"]) for r in train]).astype(np.float32))
    Y = torch.stack([r["label"] for r in train]).to(torch.float32)
    scale = float(Y.abs().max())
    X, Y = X.cuda(), (Y / scale).cuda().contiguous()
    net = nsstab.UNet(FEATURES, args.width, args.ny, args.nx, max_batch=args.batch)
    net.unet_set_params(torch.from_numpy(he_init(FEATURES, args.width, args.seed)).cuda())
    rng = np.random.default_rng(args.seed + 2)
    B = min(args.batch, len(train))
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.iters):
        idx = torch.from_numpy(rng.choice(len(train), B, replace=False)).cuda()
        lr = args.lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * k / max(1, args.iters))))
        losses.append(net.unet_train_step(X[idx].contiguous(), Y[idx].contiguous(), lr=lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    # 3. held-out pairs: Newton from the prediction vs from the plain start
    out_rows = []
    for r in test:
        st = nsstab.Stepper(Re=r["Re"], cyl_D=r["D"], **kw)
        x = torch.from_numpy(features(args.nx, args.ny, r["Re"], r["D"])[None].astype(np.float32)).cuda()
        y = torch.empty(1, args.ny, args.nx, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.unet_forward(x, y)
        q = (y[0].to(torch.float64) * scale).contiguous()
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        guess_err = float(torch.linalg.norm(q - r["label"]) / torch.linalg.norm(r["label"])) if r["ok"] else None
        rec = _solve(st, q, args)
        out_rows.append({"Re": r["Re"], "D": r["D"],
                         "plain": {k: r[k] for k in ("ok", "iters", "matvecs", "seconds", "sfd_seconds")},
                         "learned": dict(rec, inference_seconds=t_inf, guess_rel_err=guess_err)})
        del st

    def stat(key, sub):
        v = [row[key][sub] for row in out_rows if row["plain"]["ok"] and row["learned"]["ok"]]
        return float(np.mean(v)) if v else None

    if keep is not None:
        keep["net"], keep["scale"] = net, scale
    return {
        "workload": f"learned Newton start, {args.nx}x{args.ny}, Re U[{args.re_min:g},{args.re_max:g}], D U[0.8,1.2]",
        "grid": [args.nx, args.ny], "dt": dt, "T": args.T, "gmres_m": args.gmres_m, "tol": args.tol,
        "sfd_start": {"steps": args.sfd_steps, "chi": args.chi, "Delta": args.Delta},
        "train_samples": len(train), "train_requested": args.train, "test_samples": len(test),
        "unet": {"width": args.width, "params": net.count, "iters": args.iters, "batch": B, "lr": args.lr,
                 "loss_first": losses[0] if losses else None, "loss_last": float(np.mean(losses[-20:])) if losses else None,
                 "train_seconds": t_train, "storage": "bf16 activations, fp32 sums"},
        "data_seconds": t_data, "label_seconds": t_labels, "label_chains": K,
        "newton_iters_mean": {"plain": stat("plain", "iters"), "learned": stat("learned", "iters")},
        "matvecs_mean": {"plain": stat("plain", "matvecs"), "learned": stat("learned", "matvecs")},
        "newton_seconds_mean": {"plain": stat("plain", "seconds"), "learned": stat("learned", "seconds")},
        "converged": {"plain": int(sum(r["plain"]["ok"] for r in out_rows)),
                      "learned": int(sum(r["learned"]["ok"] for r in out_rows))},
        "guess_rel_err_mean": float(np.mean([r["learned"]["guess_rel_err"] for r in out_rows
                                            if r["learned"]["guess_rel_err"] is not None] or [np.nan])),
        "rows": out_rows,
        "total_seconds": time.perf_counter() - t_all,
    }


def spectral_resample(q: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """A periodic field [ny0][nx0] on a finer ny x nx grid of the same box by
    zero-padding its Fourier spectrum (the Nyquist row and column of the
    coarse grid split evenly between +k and -k), i.e. the band-limited
    interpolant sampled on the finer grid."""
    ny0, nx0 = q.shape
    F = np.fft.fft2(q) * ((ny * nx) / (ny0 * nx0))

    def maps(n0, n):
        h = n0 // 2
        src = np.r_[0:h, h, h, h + 1:n0]
        dst = np.r_[0:h, h, n - h, n - h + 1:n]
        w = np.ones(src.size)
        w[h] = w[h + 1] = 0.5
        return src, dst, w

    sr, dr, wr = maps(ny0, ny)
    sc, dc, wc = maps(nx0, nx)
    G = np.zeros((ny, nx), dtype=complex)
    R, Cc = np.meshgrid(dr, dc, indexing="ij")
    np.add.at(G, (R, Cc), F[np.ix_(sr, sc)] * wr[:, None] * wc[None, :])   # +k and -k coincide when n = n0
    return np.real(np.fft.ifft2(G))


def run_c4(args, learned: dict) -> dict:
    """The largest Newton case: 4096 x 2048, Re 100, D 1, T 1, GMRES(50), the
    FP32 propagator of the equations linearised about the current iterate as
    Jacobian, FP64 map and residual, r <= 1e-10; from the plain start (SFD
    from rest, args.c4_sfd_steps steps) and from the network's prediction at
    the training grid resampled spectrally to 4096 x 2048."""
    import torch

    nx, ny, Re, D = 4096, 2048, 100.0, 1.0
    dt = 0.01 * 128 / nx
    kw = dict(nx=nx, ny=ny, dt=dt, Re=Re, cyl_D=D)
    out = {"workload": f"Newton-Krylov base flow {nx}x{ny}, Re {Re:g}, D {D:g}, T 1, GMRES(50), tol 1e-10",
           "jacobian": "frozen (propagator of the linearised equations about the iterate), FP32"}

    def solve(q, label):
        st = nsstab.Stepper(**kw)
        lin = nsstab.Stepper(precision=32, **kw)
        _sync()
        t0 = time.perf_counter()
        rc, r, it, mv = st.newton_krylov_fixedpoint(q, T=1.0, gmres_m=50, tol=1e-10, max_newton=args.c4_max_newton,
                                                    lin=lin, jacobian="frozen")
        _sync()
        out[label] = {"status": rc, "residual": r, "newton_iters": it, "jacobian_products": mv,
                      "newton_seconds": time.perf_counter() - t0}
        print(json.dumps({"c4_" + label: out[label]}), flush=True)   # each solve as it finishes
        del st, lin
        torch.cuda.empty_cache()

    st = nsstab.Stepper(**kw)
    q = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    _sync()
    t0 = time.perf_counter()
    st.sfd_baseflow(q, chi=args.chi, Delta=args.Delta, tol=0.0, max_steps=args.c4_sfd_steps,
                    check_every=args.c4_sfd_steps)
    _sync()
    t_sfd = time.perf_counter() - t0
    r0 = st.stepper_residual(q)
    del st
    if not args.c4_skip_plain:
        solve(q, "plain")
        out["plain"].update(start=f"SFD from rest, {args.c4_sfd_steps} steps (chi {args.chi:g}, "
                                  f"Delta {args.Delta:g})", start_seconds=t_sfd, start_residual=r0)
    else:
        out["plain_start_residual"] = r0
    net, scale = learned["net"], learned["scale"]
    x = torch.from_numpy(features(args.nx, args.ny, Re, D)[None].astype(np.float32)).cuda()
    y = torch.empty(1, args.ny, args.nx, dtype=torch.float32, device="cuda")
    _sync()
    t0 = time.perf_counter()
    net.unet_forward(x, y)
    g = (y[0].to(torch.float64) * scale).cpu().numpy()
    q = torch.from_numpy(spectral_resample(g, ny, nx)).cuda()
    _sync()
    t_pred = time.perf_counter() - t0
    st = nsstab.Stepper(**kw)
    r1 = st.stepper_residual(q)
    del st
    solve(q, "learned")
    out["learned"].update(start=f"U-Net prediction at {args.nx}x{args.ny}, resampled spectrally",
                          start_seconds=t_pred, start_residual=r1)
    return out


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=64)
    ap.add_argument("--dt", type=float, default=0.0, help="time step (default 0.01 * 128 / nx)")
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--width", type=int, default=24)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--T", type=float, default=0.4)
    ap.add_argument("--gmres-m", dest="gmres_m", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-newton", dest="max_newton", type=int, default=30)
    ap.add_argument("--sfd-steps", dest="sfd_steps", type=int, default=300)
    ap.add_argument("--chi", type=float, default=0.1)
    ap.add_argument("--Delta", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--chains", type=int, default=8, help="concurrent continuation runs for the labels")
    ap.add_argument("--re-min", dest="re_min", type=float, default=40.0)
    ap.add_argument("--re-max", dest="re_max", type=float, default=150.0)
    ap.add_argument("--c4", action="store_true",
                    help="after training, the 4096x2048 Re 100 Newton solve from the plain and the learned start")
    ap.add_argument("--c4-sfd-steps", dest="c4_sfd_steps", type=int, default=400)
    ap.add_argument("--c4-max-newton", dest="c4_max_newton", type=int, default=20)
    ap.add_argument("--c4-skip-plain", dest="c4_skip_plain", action="store_true",
                    help="only the learned start of the large solve (the plain start's residual is still reported)")
    return ap.parse_args(argv)


def main(argv=None):
    from . import build

    build.build()
    args = parse(argv)
    keep = {}
    res = run(args, keep)
    # the training-grid experiment first, then (--c4) the large solve as a
    # second line, so a long run keeps what it has finished
    print(json.dumps(res), flush=True)
    if args.c4 and "net" in keep:
        print(json.dumps({"c4": run_c4(args, keep)}), flush=True)


if __name__ == "__main__":
    main()
