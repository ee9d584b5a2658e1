"""Write the oracle's reference values for the full-size water workload.

Runs the FP64 Ewald/HI oracle only (no GPU code): HI energy of all 1,000,002
atoms, dE/dlambda of all 512 sites and forces at 2,048 sampled atoms of the
seeded water system (333,334 waters, L = 21.5 nm, seed 1).  Output:
tests/golden/water_1m_seed1.json.  Takes tens of minutes on a few cores.

    python tests/golden/make_golden.py [config] [seed]
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
from oracle import hi  # noqa: E402
import synth  # noqa: E402

N_SAMPLE = 2048


def sample_atoms(n, seed):
    u = synth.uniform01(seed, 99, 4 * N_SAMPLE)
    idx = np.unique((u * n).astype(np.int64))[:N_SAMPLE]
    return idx


def input_digest(s):
    """sha256 of the generated inputs, to check that a machine regenerates them bit for bit."""
    h = hashlib.sha256()
    for k in ("x", "qA", "qB", "site_of", "lam"):
        h.update(np.ascontiguousarray(s[k]).tobytes())
    return h.hexdigest()


def main(config="C", seed=1):
    t0 = time.time()
    s = synth.make(config, seed)
    n = len(s["qA"])
    tgt = sample_atoms(n, seed)
    out = hi.hi_eval(s, targets=tgt, energy_only_full=True)
    pos = {int(i): k for k, i in enumerate(out["targets"])}
    F = np.array([out["F"][pos[int(i)]] for i in tgt])
    res = dict(
        config=config, seed=seed, n_atoms=n, L=s["L"], n_sites=len(s["lam"]),
        E=out["E"], E_qi=out["E_qi"], dEdl=out["dEdl"].tolist(), k=out["k"].tolist(),
        sample=tgt.tolist(), F=F.tolist(),
        oracle_threads=oracle.num_threads(), seconds=time.time() - t0, input_sha256=input_digest(s),
        made_by="tests/golden/make_golden.py (oracle only)",
    )
    path = os.path.join(HERE, f"water_1m_seed{seed}.json" if config == "C" else f"config{config}_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump(res, fh)
    print(path, res["seconds"])


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "C", int(sys.argv[2]) if len(sys.argv) > 2 else 1)
