"""Write tests/golden/fp64_oracle_flags.json: for every FP64 event set of the
GPU tests (tests/parity_helpers.FP64_SETS), the events on which the FP64
oracle's own |M|^2, |M'|^2, r or W' is a quarter of the FP64 bound (1e-12,
relative) or more from the extended-precision build of the same oracle.  The
GPU tests compare those events with the extended build directly.  Calls only
oracle/ and the seeded input generator.

    python tests/golden/make_fp64_oracle_flags.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2312_07440_gb300 import events as ev  # noqa: E402
from parity_helpers import FLAGS_FILE, FP64_SETS, POINT_SETS, TOL, per_event_error, set_events  # noqa: E402


def compute_flags():
    flags, worst = {}, {}
    for name, (proc, _, pts_name, _) in FP64_SETS.items():
        mom, w, ids = set_events(name)
        pts = POINT_SETS[pts_name]()
        o = oracle.reweight(proc, ev.param_vector(), pts, mom, w)
        x = oracle.reweight(proc, ev.param_vector(), pts, mom, w, precision="extended")
        err = per_event_error(o, x)
        flags[name] = [int(i) for i in ids[err >= TOL["fp64"] / 4]]
        worst[name] = float(err.max())
    return flags, worst


if __name__ == "__main__":
    flags, worst = compute_flags()
    with open(FLAGS_FILE, "w") as f:
        json.dump({"threshold": TOL["fp64"] / 4, "extended_significand_bits": oracle.extended_digits(),
                   "flags": flags, "largest_fp64_oracle_error": worst}, f, indent=1)
    print(json.dumps(flags))
