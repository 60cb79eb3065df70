"""Write ``batch_iters_seed4.json``: the constraint iteration count of every rod of the
4096-rod batch (seed 4) for which the FP64 oracle keeps every segment within 1e-3 of its
rest length (max |l / l0 - 1|, Section 2.1 "Constraints") over the 1000-step run, with a
10 % margin (the oracle must reach 0.9e-3) for the FP32 trajectory of the GPU.

Only the oracle is called.  Candidates are multiples of 10, from 10 (the paper's count).
The oracle's length error of red-black Gauss-Seidel sweeps on these hanging rods falls
roughly as 1 / n_iters, so from a rod's error at 10 iterations the smallest 10 x 2^j above
10 e_10 / (0.8 x 0.9e-3) is predicted, run, and doubled until the rod passes (error
sampled every 50 steps).  Then every count is bisected between the largest count seen to
fail and it, in multiples of 10, down to a gap of a sixteenth: the fall is not smooth (the
heaviest rod fails at 640 and reaches 0.28e-3 at 1280), and the batch's makespan is its
heaviest rods'.  Only counts that passed are kept.
Run:  python tests/golden/make_batch_iters.py  (about ten minutes on 8 cores).
"""
import dataclasses
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_04277_gb300 import workloads as W  # noqa: E402

TOL = 1e-3
ACCEPT = 0.9 * TOL
STEPS, CHUNK = 1000, 50
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_iters_seed4.json")


def max_len_err_over_run(rods):
    """Max over the run (sampled every CHUNK steps) of each rod's max |l / l0 - 1|."""
    states = [oracle.state_of(r) for r in rods]
    worst = np.zeros(len(rods))
    for _ in range(STEPS // CHUNK):
        oracle.step_batch(rods, states, CHUNK)
        for k, (r, s) in enumerate(zip(rods, states)):
            seg = np.linalg.norm(np.diff(s["pos"], axis=0), axis=1)
            worst[k] = max(worst[k], float(np.abs(seg / (r.length / (r.n_nodes - 1)) - 1.0).max()))
    return worst


def main():
    t0 = time.time()
    rods = W.batched_rods(4096, seed=4)
    iters = np.full(len(rods), 10, dtype=int)
    err = max_len_err_over_run(rods)
    err10 = err.copy()
    todo = np.nonzero(err > ACCEPT)[0]
    print(f"10 iterations: {len(todo)} of {len(rods)} rods above {ACCEPT} (worst {err.max():.3e}), "
          f"{time.time() - t0:.0f} s", flush=True)
    fail = np.zeros(len(rods), dtype=int)  # the largest count known to fail (0: none)
    fail[todo] = 10
    for k in todo:
        want = 10.0 * err[k] / (0.8 * ACCEPT)
        iters[k] = 10 * 2 ** max(1, math.ceil(math.log2(want / 10.0)))
    while len(todo):
        batch = [dataclasses.replace(rods[k], n_iters=int(iters[k])) for k in todo]
        e = max_len_err_over_run(batch)
        err[todo] = e
        bad = todo[e > ACCEPT]
        print(f"  {len(todo)} rods rerun, {len(bad)} still above, {time.time() - t0:.0f} s", flush=True)
        fail[bad] = iters[bad]
        iters[bad] *= 2
        todo = bad
    # bisection of every count between the largest count known to fail and it
    lo = np.where(fail > 0, fail, iters)
    hi = iters.copy()
    while True:
        gap = np.maximum(10, (hi // 160) * 10)
        todo = np.nonzero(hi - lo > gap)[0]
        if len(todo) == 0:
            break
        mid = np.clip(((lo[todo] + hi[todo]) // 20) * 10, lo[todo] + 10, hi[todo] - 10)
        batch = [dataclasses.replace(rods[k], n_iters=int(m)) for k, m in zip(todo, mid)]
        e = max_len_err_over_run(batch)
        ok = e <= ACCEPT
        hi[todo[ok]] = mid[ok]
        err[todo[ok]] = e[ok]
        lo[todo[~ok]] = mid[~ok]
        print(f"  bisection: {len(todo)} rods, {int(ok.sum())} passed at the midpoint, {time.time() - t0:.0f} s",
              flush=True)
    iters = hi
    out = {
        "what": "constraint iterations per rod of the 4096-rod batch (batched_rods(4096, seed=4)) for which "
                "the FP64 oracle holds max |l/l0 - 1| <= 0.9e-3 over 1000 steps (sampled every 50 steps); "
                "multiples of 10, bisected to within a sixteenth of the smallest passing count",
        "writer": "tests/golden/make_batch_iters.py (oracle only)",
        "tol": TOL, "accepted_at": ACCEPT, "steps": STEPS, "sample_every": CHUNK,
        "n_iters": [int(x) for x in iters],
        "max_len_err": [float(x) for x in err],
        "max_len_err_at_10": [float(x) for x in err10],
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    n = np.array([r.n_nodes for r in rods])
    print(f"done in {time.time() - t0:.0f} s; iterations histogram:",
          {int(v): int((iters == v).sum()) for v in np.unique(iters)},
          f"; element-iterations vs all-10: {float((n * iters).sum() / (n * 10).sum()):.2f}x")


if __name__ == "__main__":
    main()
