"""Write the FP64 oracle's answer for the full covtype-shaped workload.

The workload is ``synth.covtype_like()`` at its full size: 581,012 training
rows, d = 54 (10 dense N(0,1) columns and one-hot blocks of 4 and 40),
C = 4, gamma = 0.1, tau = 1e-3, and its 10,000 held-out rows. The script
calls only ``oracle/``:

* ``oracle.smo``: Algorithm 1 (Keerthi's modification 2, no shrinking) in
  FP64 until b_low - b_up <= 2 tau (Eq. kktterm);
* ``oracle.kkt``: f recomputed from the final alpha (Eq. fcache), the gap
  and the dual objective;
* ``oracle.decision``: Eq. (classi) before the sign on the held-out rows.

With ``--multi500`` it runs instead ``oracle.smo_shrink`` with the Table 3
policy FIXED k = 500 and multiple reconstructions (Algorithms 4-6, the
policy the benchmark times) and writes ``covtype_full_multi500*``: the GPU's
shrinking solve follows the same path, so its answer is compared with this
one at the tight tolerances, and with the unshrunk answer as a second
tau-approximate optimum.

Outputs, beside this file:

* ``covtype_full.json``: iteration count, objective, b, b_up, b_low, the
  recomputed gap, support-vector counts, a SHA-256 of alpha's bytes and of
  the generated inputs (so a test can tell a changed generator from a
  changed solver);
* ``covtype_full_decision.txt``: the 10,000 held-out decision values;
* ``covtype_full_alpha.npz``: alpha (compressed; zero for most rows).

A full run takes about 45 minutes on 6 x86 cores (340,282 steps over all
581,012 rows each; ORACLE_THREADS sets the thread count). Usage:
``python tests/golden/make_covtype_full.py``.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1406_5161_gb300 import synth  # noqa: E402


def input_digest(p) -> str:
    """SHA-256 over the generated training and held-out inputs."""
    h = hashlib.sha256()
    for a in (p.X.indptr, p.X.indices, p.X.values, p.y, p.Z.indptr, p.Z.indices,
              p.Z.values, p.yz):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


# Table 3 policy of the shrinking run: FIXED k = 500 with multiple
# reconstructions (Algorithms 4-6), the policy the benchmark uses
MULTI500 = (oracle.SHRINK_FIXED, 500, oracle.RECON_MULTI)


def main():
    threads = int(os.environ.get("ORACLE_THREADS", "0"))
    if threads > 0:
        oracle.set_threads(threads)
    shrink = "--multi500" in sys.argv
    tag = "covtype_full_multi500" if shrink else "covtype_full"
    p = synth.covtype_like()
    t0 = time.time()
    if shrink:
        r = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, *MULTI500)
    else:
        r = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    t_smo = time.time() - t0
    assert r["status"] == 0, "oracle did not converge"
    kk = oracle.kkt(p.X, p.y, r["alpha"], p.C, p.gamma)
    t1 = time.time()
    dec = oracle.decision(p.X, p.y, r["alpha"], r["b"], p.gamma, p.Z)
    t_dec = time.time() - t1
    a = r["alpha"]
    meta = {
        "workload": "covtype_like(n=581012, n_test=10000, seed=3)",
        "solver": ("oracle.smo_shrink, Table 3 FIXED k=500, multiple reconstructions" if shrink
                   else "oracle.smo (Algorithm 1, no shrinking)"),
        "shrink_events": int(r["n_shrink"]), "reconstructions": int(r["n_recon"]),
        "n": int(p.X.n), "d": int(p.X.d), "C": p.C, "gamma": p.gamma, "tau": p.tau,
        "input_sha256": input_digest(p),
        "iters": int(r["iters"]),
        "objective": r["objective"], "b": r["b"], "b_up": r["b_up"], "b_low": r["b_low"],
        "kkt_gap": kk["gap"], "kkt_objective": kk["objective"],
        "n_sv": int((a > 0).sum()), "n_bound_sv": int((a == p.C).sum()),
        "alpha_sha256": hashlib.sha256(a.tobytes()).hexdigest(),
        "held_out_positive": int((dec > 0).sum()),
        "oracle_threads": oracle.max_threads(),
        "seconds_smo": round(t_smo, 1), "seconds_decision": round(t_dec, 1),
    }
    with open(os.path.join(HERE, tag + ".json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")
    with open(os.path.join(HERE, tag + "_decision.txt"), "w") as fh:
        fh.write("# Eq. (classi) before the sign on the 10,000 held-out rows of "
                 f"covtype_like(seed=3); FP64 oracle, {meta['solver']} (make_covtype_full.py)\n")
        for v in dec:
            fh.write(f"{float(v)!r}\n")
    np.savez_compressed(os.path.join(HERE, tag + "_alpha.npz"), alpha=a)
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
