#!/usr/bin/env python3
"""Throughput of the matrix-free stability hot path on one GB300 (or N replicas).

Workload: the 2D cylinder wake at 512x256 (Re 60, dt 0.0025, sampling period
T = 0.5, i.e. 200 linearised steps per product with M = exp(T A)), Krylov
basis of dimension 128.  One bench "step" is one Krylov expansion step of
the eigen-solver: the propagator product w = M v (steps a1-a5 of the path,
200 time steps) followed by the CGS2 orthogonalisation of w against 64 basis
vectors (step a6), both through the C ABI.  The metric is grid-point time
steps per second of the linearised stepper (nx ny T/dt per step), whole job.
Also reported: the FP32 stepper on the same workload, the time to the leading
eigenvalues with Krylov-Schur (FP64 and FP32), the roofline of the dominant
kernel measured live with CUDA events, an end-to-end number through host
buffers, the SM clocks seen during the timed region, and the CPU oracle timed
on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the CPU oracle leg runs single-threaded (numpy FFT is single-threaded; pin
# BLAS too so that the reported core count is exact)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt-steps/s + time to leading eigs at 1e-8 (FP64) vs FP32/batched; % HBM roofline"
UNIT = "grid-pt-steps/s"
NX, NY = 512, 256
RE = 60.0
DT = 0.01 * 128 / NX          # CFL kept at the 128x64 value
T_SAMPLE = 0.5
KRYLOV_M = 128
BASIS_J = KRYLOV_M // 2       # basis size the timed CGS2 runs against
NEV = 8
TOL32 = 1e-6                  # Ritz residual tolerance of the FP32 eigen-solves (1e-5 eigenvalue target)
WORKLOAD = "cylinder wake 512x256, Re 60, Krylov step: M v (T=0.5, 200 linearised steps) + CGS2 vs 64 vectors"
L2_FLUSH_BYTES = 512 << 20
N_SMS = 152
FP64_FLOP_PER_CLK_SM = 4      # 2 DFMA per clock per SM: the recipe's 1.25 TFLOP/s at 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-eigs", action="store_true", help="skip the time-to-eigenvalues legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch plans (skip the autotuner)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (16 Reynolds numbers) leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg (24 solves on mixed grids)")
    ap.add_argument("--serve-grids", default="128x64,256x128,512x256",
                    help="grids the serving leg draws its solves from")
    ap.add_argument("--profile-case", default=None, metavar="NXxNY",
                    help="only run --steps linearised steps of one stepper on this grid (for ncu captures)")
    ap.add_argument("--precision", type=int, default=64, help="stepper precision of --profile-case (64, 48, 32)")
    ap.add_argument("--members", type=int, default=1, help="batch members of --profile-case")
    ap.add_argument("--fused-rows", dest="fused_rows", type=int, default=0,
                    help="--profile-case, FP32: fused row passes over strips of this many rows (0: six kernels)")
    ap.add_argument("--profile-unet", action="store_true",
                    help="only run the U-Net training leg (3 + 20 steps; for ncu launch lists)")
    ap.add_argument("--serve-c5", action="store_true",
                    help="only the serving batch on the grids {256x128 ... 2048x1024}: per-grid concurrent "
                         "batches and the persistent launch, p50/p99 for both (minutes)")
    ap.add_argument("--c1-sfd", action="store_true",
                    help="only the 128x64 case's base flow by selective frequency damping to r <= 1e-10: the "
                         "configured (chi 0.1, Delta 0.5), then Delta 2 and (chi 0.2, Delta 2), against Newton")
    ap.add_argument("--c3-full", action="store_true",
                    help="only the Reynolds sweep at 2048x1024: 16 block eigenproblems (b 8) against one plain "
                         "FP64 solve (tens of minutes)")
    return ap.parse_args()


# ------------------------------------------------------------ flop model

def fft_flops(N: int) -> int:
    """FP64 operations of one complex length-N transform as implemented:
    radix-8 passes (56 flops per butterfly, plus 7 twiddle products of 6
    flops after the first pass), then one radix-4 (16 + 3x6) or radix-2
    (4 + 6) pass."""
    logn = int(np.log2(N))
    fl, nsl = 0, 0
    while logn - nsl >= 3:
        fl += (N // 8) * (56 + (42 if nsl > 0 else 0))
        nsl += 3
    rem = logn - nsl
    if rem == 2:
        fl += (N // 4) * (16 + (18 if nsl > 0 else 0))
    elif rem == 1:
        fl += (N // 2) * (4 + (6 if nsl > 0 else 0))
    return fl


def kernel_flops(nx: int, ny: int) -> dict:
    """Algorithmic FP64 flops per launch of each step kernel (linearised step)."""
    nh = nx // 2
    rows_fft = (ny // 2) * fft_flops(nx)      # one complex transform per row pair
    cols_fft = nh * fft_flops(ny)              # one complex transform per packed column
    split = (ny // 2) * nh * 8                 # half-spectrum split / merge per pair
    return {
        "col_poisson": 2 * cols_fft + nh * ny * 3,
        "row_inverse_psi": rows_fft + (ny // 2) * nh * 4,
        "row_forward_rhs": rows_fft + split + nx * ny * 15,
        "col_update": 3 * cols_fft + nh * ny * 14,
        "row_inverse_star": ny * fft_flops(nx) + ny * nh * 4,
        "row_forward_pen": rows_fft + split + nx * ny * 20,
    }


def src_hash() -> str:
    h = hashlib.sha256()
    for f in ("stepper_impl.cuh", "fft.cuh", "common.cuh", "stepper.cuh", "df64.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1804_03859_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("src_hash") != src_hash():
        return None
    return d.get("kernels", {}).get(kernel)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------- multi-rank

def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the default process group (x itself
    when no group is initialised): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, pts_per_step: int, elapsed_max: float) -> float:
    """Whole-job grid-point steps per second: every rank runs its own replica
    of the workload (weak scaling), the job takes the slowest rank's time."""
    return world * steps * pts_per_step / elapsed_max


def share_of(items: list, rank: int, world: int) -> list:
    """Rank `rank`'s share of independent units (Reynolds numbers of a sweep,
    solves of a serving batch): every world-th one, starting at rank.  The
    units need no exchange, so the shares run with no collective."""
    return items[rank::world]


def replica_command(argv: list, gpus: int, port: int) -> list:
    """The command that runs this benchmark as `gpus` ranks of one node (one
    process per GPU) when it was started as a single process."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
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
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(nsteps_sample: int = 20, seed: int = 0):
    """Time the oracle on a bounded sample of one bench step: nsteps_sample of
    the 200 linearised steps of M v plus one CGS2 against BASIS_J vectors."""
    from oracle import ns2d
    from paper_1804_03859_gb300 import inputs

    cfg = ns2d.Config(nx=NX, ny=NY, dt=DT, Re=RE)
    base = ns2d.Base.from_omega(inputs.wake_like_field(NY, NX, seed=seed), cfg)
    v = inputs.gaussian_field(NY, NX, seed=seed + 1)
    V = np.linalg.qr(np.random.default_rng(seed).standard_normal((NX * NY, BASIS_J)))[0]
    t0 = time.perf_counter()
    w = ns2d.step_linear(v, nsteps_sample, base, cfg).ravel()
    h = V.T @ w
    w = w - V @ h
    h2 = V.T @ w
    w = w - V @ h2
    el = time.perf_counter() - t0
    return nsteps_sample * NX * NY, el


def _oracle_worker(nsteps, seed, barrier, out):
    barrier.wait()
    t0 = time.time()
    pts, _ = cpu_oracle_sample(nsteps, seed=seed)
    out.put((pts, t0, time.time()))


def cpu_oracle_all_cores(nsteps_sample: int = 10, procs: int | None = None):
    """The oracle on every host core at once: `procs` independent processes
    (spawned; numpy single-threaded in each), each running the bounded sample
    of cpu_oracle_sample on its own seed, started together.  Returns (grid-pt
    steps of all processes, wall seconds from the first start to the last
    end, processes)."""
    import multiprocessing as mpc

    procs = procs or os.cpu_count() or 1
    ctx = mpc.get_context("spawn")
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(nsteps_sample, 100 + i, barrier, q)) for i in range(procs)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    pts = sum(r[0] for r in res)
    return pts, max(r[2] for r in res) - min(r[1] for r in res), procs


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


C1 = dict(nx=128, ny=64, dt=0.01, Re=50.0, T=0.5, m=64, nev=4, tol=1e-8)


def cpu_oracle_c1_eigs(max_restarts: int = 6):
    """Time to the leading 4 eigenvalues of the 128x64 cylinder case (Re 50,
    T 0.5, Krylov-Schur m 64, tol 1e-8) with the oracle on one core, about a
    synthetic developed-wake base (inputs.wake_like_field, seed 0)."""
    from oracle import krylov, ns2d
    from paper_1804_03859_gb300 import inputs

    cfg = ns2d.Config(nx=C1["nx"], ny=C1["ny"], dt=C1["dt"], Re=C1["Re"])
    base = ns2d.Base.from_omega(inputs.wake_like_field(C1["ny"], C1["nx"], seed=0), cfg)
    v0 = inputs.gaussian_field(C1["ny"], C1["nx"], seed=1)
    mv = lambda x: ns2d.apply_expTL(base, x.reshape(C1["ny"], C1["nx"]), C1["T"], cfg).ravel()
    t0 = time.perf_counter()
    e = krylov.krylov_schur(mv, v0, m=C1["m"], nev=C1["nev"], tol=C1["tol"], max_restarts=max_restarts)
    return {"seconds": time.perf_counter() - t0, "n_matvec": e.n_matvec, "n_conv": e.n_conv,
            "n_eig": len(e.mu), "mu": [[float(m.real), float(m.imag)] for m in e.mu], "cores": 1}


def golden_c2():
    """The oracle's leading eigenvalues of the 512x256 case (written by
    tests/golden/make_c2_eigs.py), or None."""
    try:
        d = json.load(open(os.path.join(ROOT, "tests", "golden", "c2_eigs_512x256.json")))
    except Exception:
        return None
    d["mu"] = np.array([complex(a, b) for a, b in d["eigenvalues"]])
    return d


def err_vs(ref_mu, mu):
    """Relative distance of each of mu to the nearest of ref_mu."""
    return [float(np.min(np.abs(ref_mu - m)) / abs(m)) for m in mu]


# -------------------------------------------------------------- reference

def run_reference(args, rank: int):
    if rank != 0:
        return
    # W warm-up and K timed samples of the oracle
    for _ in range(args.warmup):
        cpu_oracle_sample(5)
    pts = 0
    el = 0.0
    for s in range(args.steps):
        p, e = cpu_oracle_sample(20, seed=s)
        pts += p
        el += e
    val = pts / el
    sample = f"{args.steps} samples of 20 of the 200 linearised steps of M v plus one CGS2 vs {BASIS_J} vectors, 512x256"
    out = {
        "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "grid": [NX, NY], "Re": RE, "dt": DT, "T": T_SAMPLE},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ----------------------------------------------------------------- native

def cpu_legs(args):
    """The CPU oracle timed on the host (rank 0): one core on a bounded sample
    of the bench step, every core at once (independent processes), and the
    128x64 case's time to its leading eigenvalues.  Run before any GPU work."""
    pts, el = cpu_oracle_sample(20)
    apts, ael, nproc = cpu_oracle_all_cores(10)
    c1 = cpu_oracle_c1_eigs()
    model = cpu_model()
    return {"value": pts / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "20 of the 200 linearised steps of one M v plus one CGS2 vs 64 vectors at 512x256, "
                      "numpy FP64 on one host core",
            "cpu_model": model, "cpu_count": os.cpu_count(),
            "all_cores": {"value": apts / ael, "unit": UNIT, "cores": nproc, "kind": "oracle",
                          "sample": f"{nproc} processes at once, each 10 of the 200 linearised steps of one M v "
                                    "plus one CGS2 vs 64 vectors at 512x256 (numpy FP64, one thread each)"},
            "time_to_eigs_128x64": c1}


def run_native(args, rank: int, world: int):
    cpu = cpu_legs(args) if (rank == 0 and not args.no_cpu) else None

    import torch

    from paper_1804_03859_gb300 import build, inputs, nsstab

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build() if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    nsteps = int(round(T_SAMPLE / DT))
    pts_per_step = nsteps * NX * NY
    base = torch.from_numpy(inputs.wake_like_field(NY, NX, seed=0)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    plans = {}

    def make(prec):
        st = nsstab.Stepper(nx=NX, ny=NY, dt=DT, Re=RE, precision=prec)
        if not args.no_tune:
            st.stepper_autotune(reps=5)       # project autotuner: launch plan per kernel
        plans[f"fp{prec}"] = st.plans()
        st.stepper_set_base(base)
        return st

    # basis of BASIS_J orthonormal vectors (FP64, column k contiguous)
    g = torch.Generator(device="cpu").manual_seed(1234 + rank)
    Vh = torch.linalg.qr(torch.randn(NX * NY, BASIS_J, generator=g, dtype=torch.float64))[0]
    V = Vh.T.contiguous().to(dev)
    v0 = torch.from_numpy(inputs.gaussian_field(NY, NX, seed=1)).to(dev)
    w = torch.empty_like(v0)

    def one_step(st, vin):
        st.apply_expTL(None, vin, w, T_SAMPLE)
        return nsstab.cgs2_orthogonalize(V, NX * NY, BASIS_J, w)

    def timed(st, K, W):
        for _ in range(W):
            one_step(st, v0)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        total = 0.0
        stream = torch.cuda.current_stream()
        for _ in range(K):
            flush.fill_(1.0)                                   # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(st, v0)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return max_over_ranks(total, dev) / 1e3

    st64 = make(64)
    with ClockSampler(local) as clk:
        el64 = timed(st64, args.steps, args.warmup)
    value = job_value(world, args.steps, pts_per_step, el64)

    st32 = make(32)
    el32 = timed(st32, args.steps, args.warmup)
    value32 = job_value(world, args.steps, pts_per_step, el32)

    st48 = make(48)
    el48 = timed(st48, args.steps, args.warmup)
    value48 = job_value(world, args.steps, pts_per_step, el48)

    # end to end through host buffers: H2D of v, M v + CGS2, D2H of w
    host_v = torch.from_numpy(inputs.gaussian_field(NY, NX, seed=2)).pin_memory()
    host_w = torch.empty(NY, NX, dtype=torch.float64).pin_memory()
    dv = torch.empty_like(v0)
    for _ in range(args.warmup):
        dv.copy_(host_v, non_blocking=True)
        one_step(st64, dv)
        host_w.copy_(w, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dv.copy_(host_v, non_blocking=True)
        one_step(st64, dv)
        host_w.copy_(w, non_blocking=True)
        torch.cuda.synchronize()
    e2e_el = time.perf_counter() - t0
    e2e = {"value": world * args.steps * pts_per_step / e2e_el, "unit": UNIT,
           "h2d_bytes_per_step": host_v.numel() * 8, "d2h_bytes_per_step": host_w.numel() * 8 + (BASIS_J + 1) * 8}

    # live per-kernel times of the FP64 stepper (CUDA events on its stream)
    prof_steps = nsteps
    ms = st64.stepper_profile_linear(v0, prof_steps)
    dom = max(ms, key=ms.get)
    fl = kernel_flops(NX, NY)
    dur = ms[dom] / prof_steps / 1e3
    sm_max = peaks().get("sm_max_mhz", 2070.0) or 2070.0
    peak64 = N_SMS * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12
    achieved = fl[dom] / dur / 1e12
    tr = load_traffic(dom)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s", "frac": achieved / peak64,
                "traffic": tr, "kernel": dom, "kernel_ms": ms[dom] / prof_steps,
                "flops_per_launch": fl[dom],
                "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x max SM clock (profiling recipe's 1.25 TFLOP/s)",
                "share": {k: v / sum(ms.values()) for k, v in ms.items()}}
    ms32 = st32.stepper_profile_linear(v0, prof_steps)
    ms48 = st48.stepper_profile_linear(v0, prof_steps)
    step_flops = sum(fl.values())

    # steady base flow of this workload (Newton-Krylov), about which the
    # eigen-solves below run
    newton_leg, qbase = (None, None) if (args.no_serve or args.no_eigs) else newton_leg_run(args, dev)
    eig_base = qbase if qbase is not None else base
    gold = golden_c2()

    # time to the leading eigenvalues (Krylov-Schur, m = 128, nev = 8)
    eigs = None
    if not args.no_eigs:
        eigs = {"base_flow": "Newton-Krylov steady state, r <= 1e-10" if qbase is not None else
                "synthetic developed-wake field",
                "oracle_reference": None if gold is None else
                "tests/golden/c2_eigs_512x256.json (CPU oracle: Newton base flow, Krylov-Schur m 128, tol 1e-10)"}
        ref_mu = None
        for prec, st, tol in ((64, st64, 1e-8), (48, st48, 1e-8), (32, st32, TOL32)):
            st.stepper_set_base(eig_base)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = st.arnoldi_eigs(None, v0, m=KRYLOV_M, nev=NEV, tol=tol, T=T_SAMPLE, max_restarts=8)
            el = time.perf_counter() - t0
            d = {"seconds": el, "n_matvec": r.n_matvec, "n_conv": r.n_conv, "n_eig": len(r.mu), "tol": tol,
                 "leading_mu": [r.mu[0].real, r.mu[0].imag]}
            if prec == 64:
                ref_mu = r.mu
            elif ref_mu is not None:
                d["rel_err_vs_fp64_gpu"] = err_vs(ref_mu, r.mu)
            if gold is not None and qbase is not None:
                d["rel_err_vs_oracle"] = err_vs(gold["mu"], r.mu)
            eigs[f"fp{prec}"] = d
        # the same eigenproblem with a block of 2 vectors per product with M
        # and twice the basis (block Krylov-Schur; the batched stepper runs
        # the 2 products at once)
        for prec in (64, 48):
            stb2 = nsstab.Stepper(per_set=2, nx=NX, ny=NY, dt=DT, Re=RE, precision=prec)
            if not args.no_tune:
                stb2.stepper_autotune(reps=3)
            v2 = torch.from_numpy(np.stack([inputs.gaussian_field(NY, NX, seed=400 + i) for i in range(2)])).to(dev)
            v2[0].copy_(v0)
            stb2.stepper_set_base(eig_base)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = stb2.block_arnoldi_eigs(None, v2, m=2 * KRYLOV_M, nev=NEV, tol=1e-8, T=T_SAMPLE, max_restarts=8)
            el = time.perf_counter() - t0
            d = {"seconds": el, "n_matvec": r.n_matvec, "n_conv": r.n_conv, "n_eig": len(r.mu), "tol": 1e-8,
                 "block": 2, "krylov_m": 2 * KRYLOV_M, "leading_mu": [r.mu[0].real, r.mu[0].imag]}
            if ref_mu is not None:
                d["rel_err_vs_fp64_gpu"] = err_vs(ref_mu, r.mu)
            if gold is not None and qbase is not None:
                d["rel_err_vs_oracle"] = err_vs(gold["mu"], r.mu)
            eigs[f"fp{prec}_block2"] = d
            del stb2

    # batched: 16 Reynolds numbers in 40..100 (one base flow each) stepped in
    # one launch per kernel, FP32 stepper, and their 16 eigenproblems solved
    # together by the lockstep batched Krylov-Schur driver
    batched = None
    if not args.no_batch:
        nb = 16
        Res_all = [float(x) for x in np.linspace(40.0, 100.0, nb)]
        mine = share_of(list(range(nb)), rank, world)   # this rank's Reynolds numbers (no exchange)
        Res = [Res_all[k] for k in mine]
        stb = nsstab.Stepper(nx=NX, ny=NY, dt=DT, Re=Res, precision=32)
        if not args.no_tune:
            stb.stepper_autotune(reps=3)
        bases = torch.from_numpy(np.stack([inputs.wake_like_field(NY, NX, seed=k) for k in mine])).to(dev)
        vb = torch.from_numpy(np.stack([inputs.gaussian_field(NY, NX, seed=100 + k) for k in mine])).to(dev)
        wb = torch.empty_like(vb)
        stb.stepper_set_base(bases)
        for _ in range(args.warmup):
            stb.apply_expTL(None, vb, wb, T_SAMPLE)
        torch.cuda.synchronize()
        tb = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            stb.apply_expTL(None, vb, wb, T_SAMPLE)
            e1.record()
            e1.synchronize()
            tb += e0.elapsed_time(e1) / 1e3
        tb = max_over_ranks(tb, dev)
        batched = {"members": nb, "Re": [Res_all[0], Res_all[-1]], "precision": "f32",
                   "members_per_rank": len(mine), "partition": "Reynolds numbers split across ranks, no collective",
                   "value": args.steps * nb * pts_per_step / tb, "unit": UNIT,
                   "ms_per_step": 1e3 * tb / args.steps, "plans": stb.plans()}
        if not args.no_eigs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rs = stb.batch_arnoldi_eigs(None, vb, m=KRYLOV_M, nev=NEV, tol=TOL32, T=T_SAMPLE, max_restarts=4)
            elb = time.perf_counter() - t0
            batched["time_to_eigs"] = {
                "seconds": elb, "members_converged": int(sum(r.n_conv >= len(r.mu) for r in rs)),
                "n_matvec_total": int(sum(r.n_matvec for r in rs)), "tol": TOL32,
                "sequential_estimate_seconds": (eigs or {}).get("fp32", {}).get("seconds", float("nan")) * nb,
                "sequential_estimate": "16 x the measured single-solve FP32 time above (same m, nev, tol)"}
        del stb

    # serving: 24 independent eigen-solves with grids, Reynolds numbers and
    # cylinder diameters drawn at random, run by serve_eigs (grouped by grid
    # into batched FP32 steppers, groups concurrent on their own streams)
    serving = None
    if not args.no_serve and not args.no_eigs:
        serving = serve_leg(args, dev)
    bblock = None if (args.no_batch or world > 1) else batched_block_leg(args, dev)
    unet_leg = None if args.no_serve else unet_train_leg(args, dev)
    wake_leg = None if (args.no_serve or args.no_eigs) else wake_stability_leg(args, dev)
    c1_leg = None if args.no_eigs else c1_gpu_leg(dev)

    if rank != 0:
        return
    clocks = clk.summary()
    per_step_launches = 3 + 6 * nsteps + 8   # gather, x-transform, steps, scatter; CGS2: 3 dot+reduce, 2 updates
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY], "Re": RE, "dt": DT, "T": T_SAMPLE,
                   "steps_per_matvec": nsteps, "krylov_m": KRYLOV_M, "cgs2_basis": BASIS_J,
                   "base_flow": "synthetic developed-wake field (not a converged steady state)",
                   "l2": "flushed (512 MiB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch_plans": plans},
        "roofline": roofline,
        "roofline_hbm": (bblock or {}).get("roofline_hbm"),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * per_step_launches,
        "clocks": clocks,
        "fp32": {"value": value32, "unit": UNIT, "ms_per_step": 1e3 * el32 / args.steps,
                 "kernel_ms": {k: v / prof_steps for k, v in ms32.items()}},
        "double_float": {"value": value48, "unit": UNIT, "ms_per_step": 1e3 * el48 / args.steps,
                         "dtype": "f32x2 (double-float, ~48-bit significand)",
                         "kernel_ms": {k: v / prof_steps for k, v in ms48.items()}},
        "step_flops_fp64": step_flops,
        "step_tflops_fp64": step_flops * nsteps / (el64 / args.steps) / 1e12,
        "time_to_eigs": eigs,
        "batched": batched,
        "batched_block": bblock,
        "serving": serving,
        "unet": unet_leg,
        "newton": newton_leg,
        "wake_stability": wake_leg,
        "time_to_eigs_128x64": None if c1_leg is None else {
            "workload": "cylinder 128x64, Re 50, T 0.5, Krylov-Schur m 64, leading 4 at 1e-8, synthetic wake base",
            "gpu": c1_leg, "oracle_one_core": (cpu or {}).get("time_to_eigs_128x64")},
    }
    print(json.dumps(out))


BB_SETS = 16


def batched_block_leg(args, dev, rate_grid=(2048, 1024), rate_block=8, rate_steps=40, eig_grid=(256, 128),
                      eig_block=2, eig_m=128, single_m=128, restarts=30, single_batched=True):
    """Block Krylov-Schur over a Reynolds sweep: 16 Reynolds numbers in
    40..100, each its own eigenproblem with a block of b vectors per product
    with M, FP32 stepper, all 16 b fields advanced by one launch per kernel.
    (1) Throughput of one lockstep round's product at 2048x1024 with b = 8
    (128 fields, ~268 M points per launch, far beyond L2): `rate_steps`
    linearised steps timed with CUDA events.  (2) Time to the leading 4
    eigenvalues of all 16 sets at 256x128 (tol 1e-6) with b = 2, m = 128,
    against the same 16 solves by the batched single-vector driver and
    against plain FP64 single solves run one after another (one measured,
    times 16)."""
    import torch

    from paper_1804_03859_gb300 import inputs, nsstab

    Res = [float(x) for x in np.linspace(40.0, 100.0, BB_SETS)]
    out = {"sets": BB_SETS, "Re": [Res[0], Res[-1]], "precision": "f32"}
    if rate_grid is not None:
        nx, ny = rate_grid
        dt = 0.01 * 128 / nx
        block = rate_block
        st = nsstab.Stepper(nx=nx, ny=ny, dt=dt, Re=Res, per_set=block, precision=32)
        if not args.no_tune:
            st.stepper_autotune(reps=2)
        base = torch.from_numpy(inputs.wake_like_field(ny, nx, seed=0)).to(dev)
        st.stepper_set_base(base.expand(BB_SETS, ny, nx).contiguous())
        del base
        g = torch.from_numpy(np.stack([inputs.gaussian_field(ny, nx, seed=500 + i) for i in range(block)])).to(dev)
        v = g.repeat(BB_SETS, 1, 1)
        del g
        w = torch.empty_like(v)
        T = rate_steps * dt
        st.apply_expTL(None, v, w, T)
        reps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            st.apply_expTL(None, v, w, T)
        e1.record()
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        fields = BB_SETS * block
        out["rate"] = {"grid": [nx, ny], "block": block, "fields_per_launch": fields, "steps_timed": rate_steps,
                       "reps": reps, "value": fields * nx * ny * rate_steps / sec, "unit": UNIT,
                       "ms_per_step_all_fields": 1e3 * sec / rate_steps,
                       "seconds_per_round_at_T_0_5": sec * round(0.5 / dt) / rate_steps,
                       "l2": "inputs far larger than L2 (128 fields x 2M points)", "plans": st.plans(),
                       "fused_rows": st.stepper_get_fused_rows()}
        out["roofline_hbm"] = hbm_roofline(st, v, fields * nx * ny)
        del st, v, w
        torch.cuda.empty_cache()
    if eig_grid is not None and not args.no_eigs:
        nx, ny = eig_grid
        dt = 0.01 * 128 / nx
        kw = dict(nx=nx, ny=ny, dt=dt)
        block = eig_block
        bases = torch.from_numpy(np.stack([inputs.wake_like_field(ny, nx, seed=k) for k in range(BB_SETS)])).to(dev)
        v = torch.from_numpy(np.stack([inputs.gaussian_field(ny, nx, seed=600 + i)
                                       for i in range(BB_SETS * block)])).to(dev)
        runs = {}
        stb = nsstab.Stepper(Re=Res, per_set=block, precision=32, **kw)
        if not args.no_tune:
            stb.stepper_autotune(reps=3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = stb.block_arnoldi_eigs(bases, v, m=eig_m, nev=4, tol=TOL32, T=T_SAMPLE, max_restarts=restarts)
        runs["block"] = {"seconds": time.perf_counter() - t0, "b": block, "m": eig_m,
                         "sets_converged": int(sum(r.n_conv >= len(r.mu) for r in rs)),
                         "products_total": int(sum(r.n_matvec for r in rs))}
        ref = rs
        del stb
        torch.cuda.empty_cache()
        v1 = v[::block].contiguous()
        agree = []
        if single_batched:
            sts = nsstab.Stepper(Re=Res, precision=32, **kw)
            if not args.no_tune:
                sts.stepper_autotune(reps=3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rs = sts.batch_arnoldi_eigs(bases, v1, m=single_m, nev=4, tol=TOL32, T=T_SAMPLE, max_restarts=restarts)
            runs["single_vector_batched"] = {"seconds": time.perf_counter() - t0, "m": single_m,
                                             "sets_converged": int(sum(r.n_conv >= len(r.mu) for r in rs)),
                                             "products_total": int(sum(r.n_matvec for r in rs))}
            agree = [float(max(np.min(np.abs(b.mu - x)) / abs(x) for x in a.mu)) for a, b in zip(ref, rs)
                     if a.n_conv >= len(a.mu) and b.n_conv >= len(b.mu)]
            del sts
        st64 = nsstab.Stepper(Re=Res[0], **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = st64.arnoldi_eigs(bases[0], v1[0], m=single_m, nev=4, tol=1e-8, T=T_SAMPLE, max_restarts=restarts)
        one = time.perf_counter() - t0
        runs["plain_fp64_sequential_estimate"] = {"seconds": 16 * one, "one_solve_seconds": one, "m": single_m,
                                                  "tol": 1e-8, "converged": bool(r64.n_conv >= len(r64.mu)),
                                                  "n_matvec": r64.n_matvec}
        if ref[0].n_conv >= len(ref[0].mu) and r64.n_conv >= len(r64.mu):
            runs["set0_rel_diff_block_fp32_vs_plain_fp64"] = float(
                max(np.min(np.abs(r64.mu - x)) / abs(x) for x in ref[0].mu))
        out["time_to_eigs"] = {"grid": [nx, ny], "nev": 4, "tol": TOL32, "T": T_SAMPLE, **runs,
                               "max_rel_diff_block_vs_single": max(agree) if agree else None}
    return out


ALG_BYTES_FP32_LIN = 24     # per grid-point step: read omega, N^{n-1}, Psi_b, Omega_b; write omega, N^n (FP32)


def hbm_roofline(st, v, pts: int, nsteps: int = 4):
    """HBM roofline of one linearised FP32 time step over a batch far larger
    than L2: the step's algorithmic bytes (24 B per grid point) over the
    step's live duration (CUDA events on the stepper's stream around each
    kernel, summed), against the measured copy bandwidth; with the DRAM bytes
    per grid point of the committed ncu capture of the same step, if it was
    taken on the current kernel sources."""
    ms = st.stepper_profile_linear(v, nsteps)
    step_s = sum(ms.values()) / nsteps / 1e3
    peak = peaks().get("hbm_gbs")
    achieved = ALG_BYTES_FP32_LIN * pts / step_s / 1e9
    dom = max(ms, key=ms.get)
    # DRAM bytes per grid point of one whole step, from the ncu capture of 8
    # members at 2048x1024 (each its own parameter set; here 8 members share
    # each set's base-derived fields, so the true figure is a little lower)
    tr = load_traffic("fp32_step_2048x1024_bytes_per_pt")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None,
            "traffic": None if tr is None else tr * pts,
            "traffic_bytes_per_pt": tr, "algorithmic_bytes_per_pt": ALG_BYTES_FP32_LIN,
            "dram_gbs_at_captured_traffic": None if tr is None else tr * pts / step_s / 1e9,
            "scope": "one whole linearised step (all kernels) of 128 FP32 fields at 2048x1024",
            "ms_per_step": 1e3 * step_s, "dominant_kernel": dom,
            "kernel_ms": {k: x / nsteps for k, x in ms.items()},
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, measured)"}


def newton_leg_run(args, dev):
    """Steady base flow of the bench workload (512x256, Re 60) by
    Newton-Krylov: FP64 nonlinear map and residual, Jacobian products by the
    exact tangent in FP32 arithmetic (inexact Newton), from 300 steps of
    selective frequency damping from rest."""
    import torch

    from paper_1804_03859_gb300 import nsstab

    kw = dict(nx=NX, ny=NY, dt=DT, Re=RE)
    st = nsstab.Stepper(**kw)
    lin = nsstab.Stepper(precision=32, **kw)
    q = torch.zeros(NY, NX, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.sfd_baseflow(q, chi=0.1, Delta=0.5, tol=0.0, max_steps=300, check_every=300)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    rc, r, it, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=50, tol=1e-10, max_newton=30, lin=lin)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"workload": f"steady base flow {NX}x{NY}, Re {RE}", "T": 0.4, "gmres_m": 50, "tol": 1e-10,
           "jacobian": "exact tangent (co-integrated), f32", "start": "300 SFD steps from rest (chi 0.1, Delta 0.5)",
           "status": rc, "residual": r, "newton_iters": it, "jacobian_products": mv, "sfd_seconds": t1 - t0,
           "newton_seconds": t2 - t1}
    gold = golden_c2()
    if gold is not None:
        qh = q.cpu().numpy()
        smp = gold["base_flow"]["samples"]
        out["max_sample_diff_vs_oracle"] = float(max(abs(qh[j, i] - v) for j, i, v in smp))
    return out, (q if rc == nsstab.OK else None)


def c1_gpu_leg(dev):
    """The 128x64 case's time to its leading 4 eigenvalues on the GPU (FP64
    stepper, Krylov-Schur m 64, tol 1e-8) about the same synthetic base as
    the oracle's timing in the CPU baseline, and the eigenvalues' distance
    to the oracle's."""
    import torch

    from paper_1804_03859_gb300 import inputs, nsstab

    st = nsstab.Stepper(nx=C1["nx"], ny=C1["ny"], dt=C1["dt"], Re=C1["Re"])
    base = torch.from_numpy(inputs.wake_like_field(C1["ny"], C1["nx"], seed=0)).to(dev)
    v0 = torch.from_numpy(inputs.gaussian_field(C1["ny"], C1["nx"], seed=1)).to(dev)
    st.arnoldi_eigs(base, v0, m=C1["m"], nev=C1["nev"], tol=1e-3, T=C1["T"], max_restarts=0)   # warm graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e = st.arnoldi_eigs(base, v0, m=C1["m"], nev=C1["nev"], tol=C1["tol"], T=C1["T"], max_restarts=6)
    torch.cuda.synchronize()
    return {"seconds": time.perf_counter() - t0, "n_matvec": e.n_matvec, "n_conv": e.n_conv,
            "mu": [[float(m.real), float(m.imag)] for m in e.mu], "precision": "f64"}


def wake_stability_leg(args, dev):
    """The 128x64 cylinder case end to end: for Re 40, 50, 60 the steady base
    flow by Newton-Krylov (exact tangent, from 300 SFD steps), then the
    leading eigenvalues mu of M = exp(T A) about it (Krylov-Schur, m 64,
    nev 4, tol 1e-10, T 0.5), reported as growth rate Re(log mu)/T and
    frequency Im(log mu)/T of the leading mode."""
    import torch

    from paper_1804_03859_gb300 import inputs, nsstab

    out = []
    for re in (40.0, 50.0, 60.0):
        kw = dict(nx=128, ny=64, dt=0.01, Re=re)
        st = nsstab.Stepper(**kw)
        q = torch.zeros(64, 128, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.sfd_baseflow(q, chi=0.1, Delta=0.5, tol=0.0, max_steps=300, check_every=300)
        rc, r, it, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=50, tol=1e-10, max_newton=30)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        v0 = torch.from_numpy(inputs.gaussian_field(64, 128, seed=0)).to(dev)
        e = st.arnoldi_eigs(q, v0, m=64, nev=4, tol=1e-10, T=0.5, max_restarts=40)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lam = e.growth(0.5)
        out.append({"Re": re, "base_flow": {"status": rc, "residual": r, "newton_iters": it, "seconds": t1 - t0},
                    "eigs": {"n_conv": e.n_conv, "n_matvec": e.n_matvec, "seconds": t2 - t1,
                             "mu": [[float(m.real), float(m.imag)] for m in e.mu],
                             "leading_growth_rate": float(lam[0].real), "leading_frequency": float(abs(lam[0].imag))}})
    return {"workload": "cylinder wake 128x64, dt 0.01, Re 40/50/60: Newton base flow + leading eigenvalues",
            "cases": out}


def unet_train_leg(args, dev):
    """Training-step throughput of the learned-initial-guess network
    (128x64, 3 input planes, width 24, batch 16), CUDA events on its stream."""
    import torch

    from paper_1804_03859_gb300 import learned_guess, nsstab

    ny, nx, B, width = 64, 128, 16, 24
    net = nsstab.UNet(learned_guess.FEATURES, width, ny, nx, max_batch=B)
    net.unet_set_params(torch.from_numpy(learned_guess.he_init(learned_guess.FEATURES, width, 0)).to(dev))
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal((B, learned_guess.FEATURES, ny, nx)).astype(np.float32)).to(dev)
    t = torch.from_numpy(rng.standard_normal((B, ny, nx)).astype(np.float32)).to(dev)
    for _ in range(3):
        net.unet_train_step(x, t, lr=1e-4)
    n = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(n):
        net.unet_train_step(x, t, lr=1e-4)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    fl = learned_guess.train_step_flops(learned_guess.FEATURES, width, ny, nx, B)
    bf16 = peaks().get("bf16_tflops")
    tf = fl / (ms * 1e-3) / 1e12
    return {"grid": [nx, ny], "batch": B, "width": width, "params": net.count, "ms_per_train_step": ms,
            "flops_per_step": fl, "tflops": tf, "bf16_peak_tflops": bf16,
            "frac_of_bf16_peak": tf / bf16 if bf16 else None,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 GEMM, burst)",
            "kernels": ("3x3 convolutions (forward, input and weight gradients) as implicit GEMMs on the tensor cores: "
                        "BF16 mma.sync, FP32 accumulation, FP32 gradients split bf16 hi + lo")}


SERVE_JOBS = 24
SERVE_M, SERVE_NEV, SERVE_RESTARTS = 128, 4, 8


def serve_leg(args, dev, persistent=False, grids=None):
    """Latency and throughput of serve_eigs on a seeded mixed-grid batch
    (persistent: serve_eigs_persistent, every grid in one launch per step
    kernel)."""
    import torch

    from paper_1804_03859_gb300 import inputs, nsstab

    if grids is None:
        grids = [tuple(int(x) for x in g.lower().split("x")) for g in args.serve_grids.split(",")]
    rng = np.random.default_rng(5)
    jobs = []
    for i in range(SERVE_JOBS):
        nx, ny = grids[int(rng.integers(len(grids)))]
        re, d = float(rng.uniform(40.0, 120.0)), float(rng.uniform(0.8, 1.2))
        jobs.append(dict(nx=nx, ny=ny, dt=0.01 * 128 / nx, Re=re, cyl_D=d,
                         base=torch.from_numpy(inputs.wake_like_field(ny, nx, seed=200 + i)).to(dev),
                         v0=torch.from_numpy(inputs.gaussian_field(ny, nx, seed=300 + i)).to(dev)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, res, ngroups = nsstab.serve_eigs(jobs, m=SERVE_M, nev=SERVE_NEV, tol=TOL32, T=T_SAMPLE,
                                         max_restarts=SERVE_RESTARTS, precision=32, persistent=persistent)
    wall = time.perf_counter() - t0
    lat = np.array([r["latency_s"] for r in res])
    pts = sum(r["n_matvec"] * j["nx"] * j["ny"] * round(T_SAMPLE / j["dt"]) for r, j in zip(res, jobs))
    mix = {}
    for j in jobs:
        k = f"{j['nx']}x{j['ny']}"
        mix[k] = mix.get(k, 0) + 1
    return {"form": "persistent launch over all grids" if persistent else "per-grid batches on concurrent streams",
            "solves": SERVE_JOBS, "grids": mix, "Re": [40.0, 120.0], "cyl_D": [0.8, 1.2], "precision": "f32",
            "krylov_m": SERVE_M, "nev": SERVE_NEV, "max_restarts": SERVE_RESTARTS, "tol": TOL32, "T": T_SAMPLE,
            "groups": ngroups, "status": rc, "matvecs": int(sum(r["n_matvec"] for r in res)),
            "error": nsstab.load_library().nsstab_last_error().decode() if rc < 0 else None,
            "converged": int(sum(r["status"] == nsstab.OK for r in res)),
            "wall_seconds": wall, "solves_per_s": SERVE_JOBS / wall,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max()), "min": float(lat.min())},
            "grid_pt_steps_per_s": pts / wall}


C5_GRIDS = [(256, 128), (512, 256), (1024, 512), (2048, 1024)]


def run_serve_c5(args):
    """Both serving forms on the same 24 solves drawn from the four grids."""
    import torch

    from paper_1804_03859_gb300 import build

    build.build()
    dev = torch.device("cuda")
    out = {"workload": "24 eigen-solves, grids from 256x128..2048x1024, Re U[40,120], D U[0.8,1.2], FP32, "
                       f"m {SERVE_M}, nev {SERVE_NEV}, tol {TOL32}, T {T_SAMPLE}"}
    out["concurrent_streams"] = serve_leg(args, dev, persistent=False, grids=C5_GRIDS)
    torch.cuda.empty_cache()
    out["persistent"] = serve_leg(args, dev, persistent=True, grids=C5_GRIDS)
    print(json.dumps(out))


def run_c1_sfd(args):
    """Selective frequency damping (Eq. 40) on the 128x64 cylinder case at
    Re 50 (dt 0.01) from rest to r <= 1e-10 with a step budget, with the
    configured gains and with two others; every final state against the
    Newton-Krylov base flow.  For the leading mode of this case (growth
    0.066, frequency 0.81) the closed loop (s - lam + chi)(s + 1/Delta) =
    chi/Delta has rates +0.051 (chi 0.1, Delta 0.5: unstable), -0.0038
    (Delta 2) and -0.071 (chi 0.2, Delta 2)."""
    import torch

    from paper_1804_03859_gb300 import build, inputs, nsstab

    build.build()
    kw = dict(nx=128, ny=64, dt=0.01, Re=50.0)
    st = nsstab.Stepper(**kw)
    qn = torch.zeros(64, 128, dtype=torch.float64, device="cuda")
    st.sfd_baseflow(qn, chi=0.1, Delta=0.5, tol=0.0, max_steps=300, check_every=300)
    rcn, rn, itn, _ = st.newton_krylov_fixedpoint(qn, T=0.4, gmres_m=50, tol=1e-10, max_newton=30)
    out = {"workload": "cylinder 128x64, Re 50, dt 0.01: SFD to r <= 1e-10 from rest (mirror-symmetric, so the "
                       "antisymmetric shedding mode starts at rounding level) and from rest plus 1e-3 of a seeded "
                       "Gaussian field (inputs.gaussian_field(64, 128, seed=3))",
           "newton": {"status": rcn, "residual": rn, "iters": itn}, "runs": []}
    noise = torch.from_numpy(inputs.gaussian_field(64, 128, seed=3)).cuda() * 1e-3
    for start, chi, Delta, budget in (("rest", 0.1, 0.5, 400_000), ("rest", 0.1, 2.0, 1_200_000),
                                      ("rest", 0.2, 2.0, 400_000), ("perturbed", 0.1, 0.5, 400_000),
                                      ("perturbed", 0.1, 2.0, 1_200_000), ("perturbed", 0.2, 2.0, 400_000)):
        q = torch.zeros(64, 128, dtype=torch.float64, device="cuda")
        if start == "perturbed":
            q += noise
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, r, steps = st.sfd_baseflow(q, chi=chi, Delta=Delta, tol=1e-10, max_steps=budget, check_every=2000)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        d = float(torch.max(torch.abs(q - qn)) / torch.max(torch.abs(qn))) if rcn == nsstab.OK else None
        out["runs"].append({"start": start, "chi": chi, "Delta": Delta, "step_budget": budget, "status": rc,
                            "residual": r,
                            "steps": steps, "seconds": el, "max_rel_diff_vs_newton": d})
    print(json.dumps(out))


def run_c3_full(args):
    """The Reynolds sweep at its stated size: 16 Reynolds numbers in 40..100
    at 2048x1024, each its own block eigenproblem (b 8, one synthetic wake
    base per set), FP32 stepper, against one plain FP64 single-vector solve
    at the same grid (times 16 for the sequential estimate)."""
    import torch

    from paper_1804_03859_gb300 import build

    build.build()
    dev = torch.device("cuda")
    r = batched_block_leg(args, dev, rate_grid=None, eig_grid=(2048, 1024), eig_block=8, eig_m=256,
                          single_m=128, restarts=8, single_batched=False)
    print(json.dumps(r))


def run_profile_case(args):
    """A small fixed workload for profilers: one stepper (or a batch), a
    wake-like base flow, --steps linearised steps.  Prints one line."""
    import torch

    from paper_1804_03859_gb300 import build, inputs, nsstab

    build.build()
    nx, ny = (int(x) for x in args.profile_case.lower().split("x"))
    dt = 0.01 * 128 / nx
    B = args.members
    kw = dict(nx=nx, ny=ny, dt=dt, precision=args.precision)
    st = nsstab.Stepper(Re=list(np.linspace(40.0, 100.0, B)), **kw) if B > 1 else nsstab.Stepper(Re=RE, **kw)
    shape = (B, ny, nx) if B > 1 else (ny, nx)
    base = torch.from_numpy(np.stack([inputs.wake_like_field(ny, nx, seed=k) for k in range(B)]).reshape(shape)).cuda()
    v = torch.from_numpy(np.stack([inputs.gaussian_field(ny, nx, seed=10 + k) for k in range(B)]).reshape(shape)).cuda()
    w = torch.empty_like(v)
    if args.fused_rows:
        st.stepper_set_fused_rows(args.fused_rows)
    st.stepper_set_base(base)
    st.apply_expTL(None, v, w, args.steps * dt)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "precision": args.precision, "members": B,
                      "fused_rows": st.stepper_get_fused_rows() if args.precision == 32 else 0,
                      "steps": args.steps, "max_abs": float(w.abs().max())}))


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        import socket

        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = replica_command(sys.argv[1:], args.gpus, port)
        os.execv(cmd[0], cmd)
    if args.profile_case:
        run_profile_case(args)
        return
    if args.serve_c5:
        run_serve_c5(args)
        return
    if args.c3_full:
        run_c3_full(args)
        return
    if args.c1_sfd:
        run_c1_sfd(args)
        return
    if args.profile_unet:
        import torch

        from paper_1804_03859_gb300 import build

        build.build()
        print(json.dumps(unet_train_leg(args, torch.device("cuda"))))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_native(args, rank, world)


if __name__ == "__main__":
    main()
