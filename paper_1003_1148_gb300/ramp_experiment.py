"""The integrator-accuracy experiment of Sec. IV.C on the GPU.

A Brownian particle in the harmonic potential K X^2 / 2 is driven by the ramp force
r_f t and advanced with the first-order update (Eq. 4's drift), Eq. 5 as printed, or
the complete second-order step, in FP32 with a compensated position
(``sop_brownian_ramp``). The paper's parameters, in pN, nm and ps: K = 40 pN/nm,
D = k_B T / xi = 1.5e-11 cm^2/s (1.5e-9 nm^2/ps), k_B T = 4.14 pN nm, r_f = 1e-5 pN/ns
(1e-8 pN/ps), X(0) = 0, h = 1, 25 or 50 ps, 10^9 steps, 10^5 runs.

Two measurements per (h, scheme):

* noise-free (one run): the GPU's X after n steps against the exact FP64 value of the
  scheme's recursion (its FP32 rounding error) and against Eq. 3 (the scheme's
  discretisation error plus rounding); the recursion's closed form is evaluated with
  50-digit decimals;
* with noise (n_runs runs): the mean over runs against Eq. 3, with its standard error.

Usage: ``python -m paper_1003_1148_gb300.ramp_experiment [--runs R] [--steps N]
[--h 1 25 50] [--orders 1 2 3] [--noise-free-only]``; one JSON line per measurement.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from decimal import Decimal, getcontext

KT = 4.14               # pN nm at room temperature (Sec. IV.B)
K_SP = 40.0             # pN / nm
D = 1.5e-9              # nm^2 / ps
XI = KT / D             # pN ps / nm
R_F = 1e-8              # pN / ps


def eq3(t: float, K: float = K_SP, xi: float = XI, r_f: float = R_F, X0: float = 0.0) -> float:
    """<X(t)> = X0 e^(-t/tau) + (r_f tau / xi)(t - tau (1 - e^(-t/tau))), tau = xi / K."""
    tau = xi / K
    e = math.exp(-t / tau)
    return X0 * e + r_f * tau / xi * (t - tau * (-math.expm1(-t / tau)))


def recursion_exact(n: int, h: float, order: int, K: float = K_SP, xi: float = XI, r_f: float = R_F,
                    X0: float = 0.0) -> float:
    """X_n of the noise-free scheme X_{k+1} = a X_k + b k + c (t_k = k h) in closed form,
    X_n = a^n X0 + b (a^n - n a + n - 1) / (1 - a)^2 + c (1 - a^n) / (1 - a), 50 digits."""
    getcontext().prec = 50
    K, xi, h, r_f, X0 = (Decimal(repr(v)) for v in (K, xi, h, r_f, X0))
    tau = xi / K
    a = 1 - h / tau
    b = r_f * h * h / xi
    c = Decimal(0)
    if order >= 2:
        a += h * h / (2 * tau * tau)
        b *= 1 - h / (2 * tau)
    if order == 3:
        c = r_f * h * h / (2 * xi)
    an = (Decimal(n) * a.ln()).exp()
    return float(an * X0 + b * (an - n * a + n - 1) / (1 - a) ** 2 + c * (1 - an) / (1 - a))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--runs", type=int, default=100_000)
    ap.add_argument("--steps", type=int, default=1_000_000_000)
    ap.add_argument("--noise-free-steps", type=int, default=None)
    ap.add_argument("--h", type=float, nargs="+", default=[1.0, 25.0, 50.0])
    ap.add_argument("--orders", type=int, nargs="+", default=[1, 2, 3])
    ap.add_argument("--noise-free-only", action="store_true")
    ap.add_argument("--seed", type=int, default=2010)
    args = ap.parse_args(argv)
    from . import sop
    nf_steps = args.noise_free_steps or args.steps
    for h in args.h:
        for order in args.orders:
            t0 = time.perf_counter()
            mean, _ = sop.brownian_ramp(K_SP, XI, 0.0, h, R_F, 1, nf_steps, order=order, n_out=1)
            wall = time.perf_counter() - t0
            x_gpu, x_rec, x_th = float(mean[0]), recursion_exact(nf_steps, h, order), eq3(nf_steps * h)
            print(json.dumps({"experiment": "noise-free", "h_ps": h, "order": order, "steps": nf_steps,
                              "t_ps": nf_steps * h, "x_gpu_nm": x_gpu, "x_recursion_nm": x_rec, "x_eq3_nm": x_th,
                              "rel_err_gpu_vs_recursion": abs(x_gpu - x_rec) / abs(x_rec),
                              "rel_err_recursion_vs_eq3": abs(x_rec - x_th) / abs(x_th),
                              "rel_err_gpu_vs_eq3": abs(x_gpu - x_th) / abs(x_th), "wall_s": wall}), flush=True)
    if args.noise_free_only:
        return 0
    for h in args.h:
        for order in args.orders:
            t0 = time.perf_counter()
            mean, var = sop.brownian_ramp(K_SP, XI, KT, h, R_F, args.runs, args.steps, order=order, n_out=1,
                                          seed=args.seed)
            wall = time.perf_counter() - t0
            m, se, x_th = float(mean[0]), math.sqrt(float(var[0]) / args.runs), eq3(args.steps * h)
            print(json.dumps({"experiment": "stochastic", "h_ps": h, "order": order, "runs": args.runs,
                              "steps": args.steps, "t_ps": args.steps * h, "mean_nm": m, "se_nm": se,
                              "x_eq3_nm": x_th, "rel_err_vs_eq3": abs(m - x_th) / abs(x_th),
                              "rel_se": se / abs(x_th), "z": (m - x_th) / se if se > 0 else None,
                              "run_steps_per_s": args.runs * args.steps / wall, "wall_s": wall}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
