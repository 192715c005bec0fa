"""Writes ``config4_oracle.json``: the CPU oracle on the Q1 elasticity
workload of the benchmark's 32-right-hand-side form
(``awg_inputs.config4()``: 384 x 384 elements, left edge clamped, layered
Young's modulus 1 / 1e5, 16 x 16 node boxes, overlap 2, tau = 0.1), for the
full-size parity test of that workload.  Calls only ``oracle`` and the
input generators; about half an hour on eight cores.

    python tests/golden/make_config4_reference.py

Stored: the per-subdomain counts n^s_-, strictly negative counts and GenEO
mode counts (all 256 subdomains); n0 and n_-; the smallest relative
distance of a GenEO pencil eigenvalue to tau; max_s cond(A^s_+); the PCG
iteration counts and true relative residuals of H_3,ad (rtol 1e-8) on
columns 0, 1, 16 and 31 of the workload's 32 right-hand sides; 4096
sampled entries of H_3,ad x for x ~ N(0,1) from default_rng(4242), with the
2-norm and the largest magnitude of the whole H_3,ad x.
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import awg_inputs as gi  # noqa: E402
import oracle as O  # noqa: E402


def main():
    t0 = time.time()
    p = gi.config4()
    st = O.setup_problem(p)
    mm = O.minus_counts(st)
    gap = min(float(np.min(np.abs(lam - st.tau))) / st.tau for lam in st.geneo_lam)
    cols = {}
    for c in (0, 1, 16, 31):
        rc = O.pcg(lambda v: st.A @ v, p.b[c], lambda r: O.H3_ad_apply(st, r), rtol=1e-8)
        cols[str(c)] = {"iters": int(rc.iters), "true_relres": float(rc.true_relres)}
    x = np.random.default_rng(4242).standard_normal(p.n)
    y = O.H3_ad_apply(st, x)
    idx = np.sort(np.random.default_rng(4243).choice(p.n, 4096, replace=False))
    out = {
        "source": "oracle/awg_oracle.py on awg_inputs.config4() (Q1 elasticity 384 x 384, layered E 1 / 1e5, "
                  "256 node boxes, overlap 2, tau = 0.1, 32 right-hand sides), written by "
                  "tests/golden/make_config4_reference.py",
        "n": int(p.n), "n0": int(st.n0), "n_minus": int(st.n_minus),
        "n_minus_per_subdomain": mm[:, 0].tolist(), "n_strict_per_subdomain": mm[:, 1].tolist(),
        "modes_per_subdomain": O.mode_counts(st).tolist(),
        "geneo_min_rel_gap_to_tau": gap,
        "local_condition": O.local_condition(st),
        "pcg_columns": cols,
        "apply_h3ad": {"x_seed": 4242, "idx_seed": 4243, "idx": idx.tolist(), "y": y[idx].tolist(),
                       "y_max_abs": float(np.abs(y).max()), "y_norm": float(np.linalg.norm(y))},
        "seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config4_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
