"""Writes c2_oracle_timing.json: the measured wall time of the whole oracle
IPN solve of the 3D benchmark instance stored in c2_ipn_oracle.npz, next to
what the oracle's timing model (oracle.timing.projection) projects for the
same solve (same iteration counts) on the same machine.  Their ratio
calibrates the model wherever it is used for a baseline.  Run it on the
machine that ran make_c2_ipn_oracle.py, with nothing else running.  Calls
only the oracle.

    python tests/golden/calibrate_c2_oracle_model.py
"""
import json
import os
import platform
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rfm_workloads as W  # noqa: E402
from oracle import timing  # noqa: E402


def main():
    ref = np.load(os.path.join(HERE, "c2_ipn_oracle.npz"))
    it, ls = int(ref["outer_iters"]), int(np.sum(ref["lsqr_iters"]))
    per, sample, spent = timing.projection(W.config_c2(), W.opts_c2(), it, ls)
    out = {"measured_wall_s": float(ref["wall_s"]), "projected_s": per, "outer_iters": it, "lsqr_iters": ls,
           "cores": int(ref["cores"]), "workers": int(ref["workers"]), "cpu": str(ref["cpu"]),
           "machine": str(ref["machine"]), "model_sample": sample}
    assert platform.machine() == out["machine"], "run on the machine that measured the solve"
    with open(os.path.join(HERE, "c2_oracle_timing.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
