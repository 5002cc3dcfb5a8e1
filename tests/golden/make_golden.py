"""Writes oracle_fixtures.json: stored outputs of the FP64 oracle on small
seeded inputs, a regression record of the oracle's arithmetic, and a digest
of every synthetic workload the benchmark and the tests use.

The paper prints no worked example with numbers, so these values are not
the paper's: each is written by this script, which calls only the oracle and
the seeded input generators.  They are not pins (the pins check the oracle
against closed forms, quadrature, finite differences and invariants); they
make any later change to the oracle's results visible, since the fixture
must then be rewritten by this script in the same commit.

    python tests/golden/make_golden.py          # rewrite the fixture
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import scenes  # noqa: E402

FIXTURE = os.path.join(HERE, "oracle_fixtures.json")

# a fixed pose off the optimum: T = exp(xi^), xi = (omega, v)
XI = [0.03, -0.02, 0.05, 0.04, -0.03, 0.02]

CASES = [
    {"name": "cube-800 dense, RGB block",
     "cite": "Eq. (double_sum) with Eq. (k) and the colour kernel of Eq. (newscalar); gradient and second "
             "derivative of the left-perturbed pose (the gradient ascent on SE(3) of Sec. I)",
     "kind": "evaluate", "scene": "cube", "n": 800, "seed": 2101,
     "kw": {"ell": 0.2, "cutoff_mult": 0.0}},
    {"name": "semantic-3000 cutoff 3 l, RGB + 19 labels",
     "cite": "Eq. (double_sum) over the pairs within 3 l (Sec. III-B sparsity); labels by the inner product "
             "of Eq. (scalar), tensor product of Eq. (tensor_product)",
     "kind": "evaluate", "scene": "batch", "n": 3000, "seed": 2102,
     "kw": {"ell": 0.3, "cutoff_mult": 3.0}},
    {"name": "semantic-3000 cutoff 3 l with the feature cutoff 1.6",
     "cite": "as above, with the optional feature-space cutoff (Sec. III-B)",
     "kind": "evaluate", "scene": "batch", "n": 3000, "seed": 2102,
     "kw": {"ell": 0.3, "cutoff_mult": 3.0, "feat_cutoff_mult": 1.6}},
    {"name": "cube-800 indicator and cosine",
     "cite": "Eq. (indicator_actual) and Eq. (indicator) of Sec. III-C",
     "kind": "indicator", "scene": "cube", "n": 800, "seed": 2101,
     "kw": {"ell": 0.2, "cutoff_mult": 3.0}},
    {"name": "cube-800 input gradients",
     "cite": "derivatives of Eq. (double_sum) in the points, features and l, pair set held fixed (Sec. VI's "
             "learned features)",
     "kind": "backward", "scene": "cube", "n": 800, "seed": 2101,
     "kw": {"ell": 0.2, "cutoff_mult": 3.0}},
    {"name": "cube-600 registration, 12 iterations",
     "cite": "gradient ascent on SE(3) with the line-Newton step and the exponential update (Sec. I, Sec. III)",
     "kind": "register", "scene": "cube", "n": 600, "seed": 2103,
     "kw": {"ell": 0.15, "cutoff_mult": 3.0, "max_iters": 12, "step_tol_rot": 0.0, "step_tol_trans": 0.0}},
]


# The benchmark's and the tests' synthetic workloads, recorded by a digest of
# every array they hold, so that a change to a generator (or to the random
# streams it draws from) cannot silently change a measured workload.
SCENES = {
    "cube-2000": lambda: [scenes.cube_pair()],
    "street-20k": lambda: [scenes.street_pair()],
    "room-19k": lambda: [scenes.room_pair()],
    "batch-64": lambda: scenes.batch_pairs(),
    "box80-200k": lambda: [scenes.large_pair()],
}


def scene_digest(name):
    h = hashlib.sha256()
    pairs = SCENES[name]()
    points = 0
    for p in pairs:
        for a in (p.X, p.Z, p.FX, p.FZ):
            a = np.ascontiguousarray(a, dtype=np.float32)
            h.update(str(a.shape).encode())
            h.update(a.tobytes())
        h.update(np.ascontiguousarray(p.T_true, dtype=np.float64).tobytes())
        h.update(repr((p.blocks, sorted(p.params.items()))).encode())
        points += p.n + p.m
    return {"pairs": len(pairs), "points": points, "sha256": h.hexdigest()}


def inputs(case):
    if case["scene"] == "cube":
        p = scenes.cube_pair(n=case["n"], seed=case["seed"])
    else:
        n = case["n"]
        p = scenes.batch_pairs(n_pairs=1, seed=case["seed"], n_range=(n, n))[0]
    return p


def compute(case):
    p = inputs(case)
    kw = dict(case["kw"])
    T = oracle.se3_exp(np.array(XI))
    feats = dict(FX=p.FX, FZ=p.FZ, blocks=p.blocks)
    if case["kind"] == "evaluate":
        e = oracle.evaluate(p.X, p.Z, T, **feats, **kw)
        e2 = oracle.evaluate(p.X, p.Z, T, direction=e["g"], **feats, **kw)
        return {"F": e["F"], "grad": list(e["g"]), "Fpp_along_grad": e2["Fpp"], "npairs": e["npairs"]}
    if case["kind"] == "indicator":
        return {"i_theta": oracle.indicator(p.X, p.Z, T, **feats, **kw),
                "cosine": oracle.cosine(p.X, p.Z, T, FX=p.FX, FZ=p.FZ, blocks=p.blocks, **kw)}
    if case["kind"] == "backward":
        b = oracle.backward(p.X, p.Z, T, **feats, **kw)
        return {"dell": float(b["dell"]), "dX_rows_0_4": b["dX"][:5].tolist(), "dZ_rows_0_4": b["dZ"][:5].tolist(),
                "dFX_row_0": b["dFX"][0].tolist(), "dFZ_row_0": b["dFZ"][0].tolist()}
    if case["kind"] == "register":
        Tout, info, tr = oracle.register(p.X, p.Z, np.eye(4), **feats, **kw)
        return {"T_out": Tout.tolist(), "F_per_iter": tr[:, 1].tolist(), "iters": info["iters"]}
    raise ValueError(case["kind"])


def main():
    out = {"about": "FP64 oracle outputs on seeded synthetic inputs (a regression record; not the paper's "
                    "numbers, which it does not print). Pose T = exp(xi^) with xi = (omega, v).",
           "generator": "python tests/golden/make_golden.py",
           "xi": XI,
           "cases": [dict(c, expected=compute(c)) for c in CASES],
           "scenes": {name: scene_digest(name) for name in SCENES}}
    with open(FIXTURE, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
