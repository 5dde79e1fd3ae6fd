"""Write tests/golden/plummer4096_oracle.json from the CPU oracle alone.

The workload is the N = 4096 equal-mass Plummer sphere in Henon units
(theta = 0.5, quadrupole, r_out = 0.05, r_in = 0.1 r_out, dt = 1/256).  The
file pins the oracle against later drift: any change to its arithmetic that
moves these numbers has to name the passage of the paper that justifies it.
Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    c = synth.plummer(4096, synth.BASE_SEED)
    t = oracle.Tree(c.x, c.y, c.z, c.m, theta=0.5, r_out=0.05, leaf_cap=16, group_size=64)
    d = t.export()
    f = t.far(0.005)
    counts, offs, idx = t.neighbours(0.05)
    vx, vy, vz = oracle.kick(1.0 / 256, f["a"][:, 0], f["a"][:, 1], f["a"][:, 2], c.vx, c.vy, c.vz)
    out = {
        "workload": "plummer N=4096 equal masses seed=20211022 theta=0.5 r_out=0.05 r_in=0.005 "
                    "leaf_cap=16 group_size=64 quadrupole dt=1/256",
        "keys_sha256": hashlib.sha256(d["keys"].tobytes()).hexdigest(),
        "perm_sha256": hashlib.sha256(d["perm"].tobytes()).hexdigest(),
        "n_nodes": t.n_nodes, "n_groups": t.n_groups, "depth": int(d["level"].max()),
        "n_cell_total": int(f["n_cell"].sum()), "n_part_total": int(f["n_part"].sum()),
        "nbr_total": int(offs[-1]),
        "nbr_sha256": hashlib.sha256(idx.tobytes()).hexdigest(),
        "a_far_first8": f["a"][:8].tolist(),
        "pot_first8": f["pot"][:8].tolist(),
        "v_kicked_first4": np.stack([vx[:4], vy[:4], vz[:4]], 1).tolist(),
    }
    with open(os.path.join(HERE, "plummer4096_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
