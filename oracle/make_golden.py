"""Write tests/golden/energies.json: the oracle's ladder energy E_L for the
seeded workloads (R = ladder(L, t2) from R = 0).

TEST INFRASTRUCTURE: calls only the CPU oracle and the seeded generators.
Usage: python -m oracle.make_golden c1 c2 [c3]   (c2 ~ 2 min, c3 ~ 1 h on 8 cores)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from ladder_inputs import CONFIGS, make_inputs  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "energies.json")


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        s = CONFIGS[name]
        L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
        t0 = time.time()
        R = oracle.ladder(L, t2)
        E = oracle.energy(t2, R)
        data[name] = {
            "no": s.no, "nv": s.nv, "nchol": s.nchol, "seed": s.seed, "E_L": E,
            "R_fro": float((R * R).sum() ** 0.5),
            "source": "oracle.ladder + oracle.energy (plain FP64 loops, Eq. vfunction-chol; "
                      "E_L = sum (2 t_ij^ab - t_ij^ba) R_ij^ab) on ladder_inputs.make_inputs",
            "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.num_threads(),
        }
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c2"])
