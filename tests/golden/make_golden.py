"""Write tests/golden/small_workload.json: SHA-256 digests of the seeded small
workload's uint8 input and of the oracle's (DM,t) plane for it, plus a few
plane values.

Calls only the oracle and the seeded generator; run from the repository root:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import filterbank as fb  # noqa: E402
import oracle  # noqa: E402


def small_case():
    w = fb.SMALL
    table = oracle.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms = w.dm_list()
    S = oracle.maxshift(table, dms)
    pulses = fb.all_pulses(w)
    delays = [np.array([oracle.shift(p.dm, table[c]) for c in range(w.nchan)]) for p in pulses]
    data = fb.filterbank(w.nchan, w.nsamp_out + S, w.seed, pulses, delays)
    return w, table, dms, S, data


def main():
    w, table, dms, S, data = small_case()
    plane = oracle.dedisperse(data, table, dms, w.nsamp_out)
    rec = {
        "workload": w.name,
        "maxshift": S,
        "input_sha256": hashlib.sha256(data.tobytes()).hexdigest(),
        "dmshift_sha256": hashlib.sha256(table.tobytes()).hexdigest(),
        "plane_sha256": hashlib.sha256(plane.tobytes()).hexdigest(),
        "plane_samples": {f"{d},{t}": float(plane[d, t])
                          for d, t in [(0, 0), (30, 2000), (30, 2003), (63, 8191), (17, 4321)]},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_workload.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
