"""Write the oracle's record of one zero-beta step at full size (tests/golden/*.json).

Calls only the CPU oracle and the seeded input generator. The record holds the step
coefficients, the PCG iteration counts and residuals, per-field L2 norms and the oracle's values
at seeded sample positions (sample_index regenerates them: 20,000 per field, a quarter of them on
the rows every boundary rule acts on: the two polar rows, and the rows next to them for B_theta,
and the first and last radial layers). It serves the full-size GPU parity test (sampled outputs)
and gives the CPU baseline the oracle's own iteration counts at this size.

    python tests/golden/make_golden.py fluxrope_256x256x512          # PC1 (point Jacobi)
    python tests/golden/make_golden.py fluxrope_256x256x512 --pc2    # PC2 (phi-line ILU(0))
    python tests/golden/make_golden.py fluxrope_256x256x512 --pc2 --sts   # PC2, RKL2 viscosity
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1811_02605_gb300 import inputs as I  # noqa: E402

NSAMPLE = 20000


def sample_index(shape, seed):
    """Sorted flat indices into an array of `shape` (nr', nt', np): three quarters drawn from the
    whole array, one quarter from the boundary rows (theta rows 0, 1, nt'-2, nt'-1 and radial
    layers 0 and nr'-1)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    a, b, c = shape
    m = min(NSAMPLE, n)
    rows = sorted({0, 1, b - 2, b - 1} & set(range(b)))
    edge = [(i * b + j) * c + np.arange(c) for i in range(a) for j in rows]
    edge += [(i * b + j) * c + np.arange(c) for i in sorted({0, a - 1}) for j in range(b) if j not in rows]
    edge = np.unique(np.concatenate(edge))
    pick_edge = rng.choice(edge, size=min(m // 4, edge.size), replace=False)
    rest = rng.choice(n, size=m - pick_edge.size, replace=False)
    return np.unique(np.concatenate([pick_edge, rest]))


def main(name, pc2=False, sts=False):
    w, st = I.workload(name)
    d = w["desc"]
    g = O.Grid.from_desc(d)
    t0 = time.time()
    out, info = g.step(st, nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=w["tol"], pc2=pc2, sts=sts)
    wall = time.time() - t0
    rec = dict(workload=name, desc=dict(nr=d.nr, nt=d.nt, np=d.np, r0=d.r0, r1=d.r1, stretch=d.stretch),
               params=dict(nu=w["nu"], eta=w["eta"], cfl=w["cfl"], tol=w["tol"], preconditioner=1 if pc2 else 0,
                           viscosity_sts=1 if sts else 0),
               info={k: (v if not isinstance(v, np.floating) else float(v)) for k, v in info.items()},
               oracle_step_seconds=wall, fields={})
    rec["info"] = {k: ([float(x) for x in v] if isinstance(v, list) else float(v)) for k, v in info.items()}
    for k, a in out.items():
        idx = sample_index(a.shape, sum(map(ord, k)) + 7)
        rec["fields"][k] = dict(shape=list(a.shape), l2=float(np.linalg.norm(a)),
                                l2_initial=float(np.linalg.norm(st[k])),
                                sample_seed=sum(map(ord, k)) + 7, sample=a.ravel()[idx].tolist())
    tag = ("_pc2" if pc2 else "") + ("_sts" if sts else "")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle{tag}_step1.json")
    with open(path, "w") as f:
        json.dump(rec, f)
    print(path, rec["info"], wall)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    main(args[0] if args else "fluxrope_256x256x512", pc2="--pc2" in sys.argv, sts="--sts" in sys.argv)
