"""Writes full_size_solutions.json: the FP64 oracle's solutions of the two
full-size noisy workloads, as values at a fixed sample of indices.

Workloads: the hyperspectral-shaped tensor (256 x 256 x 128, TT-ranks
(1,20,20,1), 838 861 observed entries, N(0, 1e-3^2) noise) and the
tomography-shaped tensor (order 12, mode size 4, interior TT-rank 8, 2e5
entries, N(0, 1e-4^2) noise), seed 0 of each (paper_2501_13385_gb300.workloads).

Solver: the plain FP64 CPU PRGD of oracle/ (Algorithm 2), eps_rel 1, stopped
by the rule of the paper's noise experiment (Section 5):
||T_{l+1} - T_l||_F <= 1e-5 max(1, ||T_l||_F).  Step sizes: the steepest
step of Eq. (PRGD stepsize) for the hyperspectral shape (the constant form of
Theorem 4.1 with alpha_scale 1.5 diverges there, and 0.5 converges ~10x
slower), the constant form with alpha_scale 1.5 for the tomography shape.
The oracle is run one iteration past its stop so that iterates stop-1, stop and stop+1 are
all recorded (a run that stops one iteration earlier or later is compared
with the matching iterate).

Stored per workload: the stop iteration, the sample indices (512 uniform
draws of multi-indices, numpy default_rng(20250123), with replacement), and
for each of the three iterates its values at the samples and its Frobenius
norm.  The estimate sqrt(sum diff^2 / sum ref^2) over the samples is an
unbiased stand-in for the relative Frobenius distance of two tensors.

Only oracle/ and the workload generators are used; nothing here calls the
CUDA library.  Runtime: several minutes per workload on one CPU core.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_2501_13385_gb300 import workloads as w  # noqa: E402

TOL = 1e-5
SAMPLES = 512


STEP = {"hyperspectral_like": "adaptive", "tomography_like": "constant"}


def solve_with_neighbours(P, step_rule):
    cur = [np.array(c) for c in P.init]
    iterates = []
    stop = None
    for it in range(1, 401):
        new, _ = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5, step=step_rule)
        change = o.tt_dist(new, cur) / max(1.0, o.tt_norm(cur))
        iterates.append(new)
        iterates = iterates[-3:]
        cur = new
        if stop is None and change <= TOL:
            stop = it
        if stop is not None and it == stop + 1:
            return stop, iterates
        print(f"  iteration {it}: step change {change:.3e}", flush=True)
    raise RuntimeError("oracle did not reach the stop rule")


def main():
    out = {}
    for name in ("hyperspectral_like", "tomography_like"):
        P = getattr(w, name)(0)
        print(name, flush=True)
        stop, its = solve_with_neighbours(P, STEP[name])
        rng = np.random.default_rng(20250123)
        sidx = np.stack([rng.integers(0, nk, SAMPLES) for nk in P.n], axis=1)
        out[name] = {
            "seed": 0, "n": P.n, "r": P.r, "stop_rule": "step", "tol": TOL, "stop": stop,
            "step": STEP[name], "alpha_scale": 1.5,
            "idx": sidx.astype(int).tolist(),
            "iterates": {str(stop - 1 + j): {"values": [float(v) for v in o.tt_eval(c, sidx)],
                                             "norm": o.tt_norm(c)} for j, c in enumerate(its)},
            "relerr_vs_truth": o.tt_dist(its[1], P.truth) / o.tt_norm(P.truth),
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_solutions.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", path)


if __name__ == "__main__":
    main()
