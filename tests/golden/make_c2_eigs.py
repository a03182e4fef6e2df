"""Write tests/golden/c2_eigs_512x256.json from the CPU oracle alone.

The cylinder wake on the 512x256 grid at Re 60 (dt 0.0025, the 128x64
case's CFL): its steady base flow and the leading eigenvalues of the
propagator M = exp(T A) about it, T = 0.5, by Krylov-Schur with a basis of
128 vectors (Sec. 3.2.2), 8 leading values.

Recipe (the GPU test repeats it with the library):
  1. 300 steps of selective frequency damping (Eq. 40, chi 0.1, Delta 0.5)
     from rest (omega = 0);
  2. Newton-Krylov (Sec. 3.1.2, Eq. 43) on Phi_T, T = 0.4, GMRES(50),
     stopped at r(q) <= 1e-10 (Sec. 3.1.4's target), Jacobian = the
     linearised propagator about the current iterate (exact at the fixed
     point, which is all the converged base flow depends on);
  3. Krylov-Schur, m = 128, nev = 8, |b^T y| <= 1e-10 (Eq. 63), start
     vector inputs.gaussian_field(256, 512, seed=1).

Only oracle/ and the seeded input generator are called.  About two hours of
one CPU core.  Usage:

    python tests/golden/make_c2_eigs.py [--cache BASE.npy]

--cache keeps the base flow between runs (read if present, else written).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, newton, ns2d, sfd  # noqa: E402
from paper_1804_03859_gb300 import inputs  # noqa: E402

NX, NY, RE = 512, 256, 60.0
DT = 0.01 * 128 / NX
T_NEWTON, T_EIG = 0.4, 0.5
M, NEV, TOL = 128, 8, 1e-10
# fixed sample points (j, i) of the base flow: near the cylinder, in the wake, in the fringe
SAMPLES = [(128, 128), (120, 136), (136, 136), (128, 160), (112, 200), (144, 200), (128, 300), (100, 400),
           (156, 400), (128, 470), (64, 64), (200, 250), (128, 120), (130, 140), (126, 140), (10, 10)]
OUT = os.path.join(ROOT, "tests", "golden", "c2_eigs_512x256.json")


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def base_flow(cfg):
    q = np.zeros((NY, NX))
    q, r_sfd, _, _ = sfd.sfd_baseflow(cfg, q, chi=0.1, Delta=0.5, tol=0.0, max_steps=300, check_every=300)
    log(f"SFD 300 steps: r = {r_sfd:.3e}")
    t0 = time.perf_counter()
    res = newton.newton_baseflow(cfg, q, T=T_NEWTON, tol=1e-10, max_newton=30, m=50, jacobian="frozen")
    log(f"Newton: r = {res.residual:.3e}, {res.iters} iterations, {res.matvecs} products, "
        f"{time.perf_counter() - t0:.0f} s")
    if not res.converged:
        raise SystemExit("Newton did not reach r <= 1e-10")
    return res.x, res.residual, res.iters, res.matvecs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None)
    args = ap.parse_args()
    cfg = ns2d.Config(nx=NX, ny=NY, dt=DT, Re=RE)
    t_start = time.perf_counter()
    if args.cache and os.path.exists(args.cache):
        qb = np.load(args.cache)
        nit = nmv_newton = None
        log(f"base flow from {args.cache}")
    else:
        qb, _, nit, nmv_newton = base_flow(cfg)
        if args.cache:
            np.save(args.cache, qb)
    r = ns2d.residual(qb, cfg)
    base = ns2d.Base.from_omega(qb, cfg)
    count = [0]

    def matvec(x):
        count[0] += 1
        if count[0] % 25 == 0:
            log(f"product {count[0]}")
        return ns2d.apply_expTL(base, x.reshape(NY, NX), T_EIG, cfg).ravel()

    v0 = inputs.gaussian_field(NY, NX, seed=1)
    t0 = time.perf_counter()
    e = krylov.krylov_schur(matvec, v0, m=M, nev=NEV, tol=TOL, max_restarts=40)
    log(f"Krylov-Schur: {e.n_conv}/{len(e.mu)} converged, {e.n_matvec} products, {e.restarts} restarts, "
        f"{time.perf_counter() - t0:.0f} s")
    mirror = qb[::-1, :]
    mirror = np.roll(mirror, 1, axis=0)   # y -> Ly - y on the vertex grid: j -> (ny - j) mod ny
    lam = np.log(e.mu.astype(complex)) / T_EIG
    out = {
        "citation": ("Sec. 3.2.2 (Krylov-Schur, Eqs. 60-63) on the propagator of Eq. 42 about the steady base "
                     "flow of Sec. 3.1.2 (Newton, Eq. 43) at r <= 1e-10 (Sec. 3.1.4); written by "
                     "tests/golden/make_c2_eigs.py from oracle/ alone"),
        "grid": [NX, NY], "Re": RE, "dt": DT, "T": T_EIG, "krylov_m": M, "nev": NEV, "tol": TOL,
        "start_vector": "inputs.gaussian_field(256, 512, seed=1)",
        "base_flow": {
            "recipe": "300 SFD steps (chi 0.1, Delta 0.5) from rest, then Newton-Krylov T 0.4, GMRES(50), "
                      "r <= 1e-10",
            "residual": r, "newton_iters": nit, "newton_products": nmv_newton,
            "norm_h": float(ns2d.norm_h(qb, cfg)), "max_abs": float(np.abs(qb).max()),
            "mirror_antisymmetry_defect": float(np.abs(qb + mirror).max()),
            "samples": [[j, i, float(qb[j, i])] for j, i in SAMPLES],
        },
        "eigenvalues": [[float(m.real), float(m.imag)] for m in e.mu],
        "residuals": [float(x) for x in e.residual],
        "growth_rates": [float(x.real) for x in lam],
        "frequencies": [float(x.imag) for x in lam],
        "n_conv": e.n_conv, "n_matvec": e.n_matvec, "restarts": e.restarts,
        "cpu_seconds": time.perf_counter() - t_start,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()
