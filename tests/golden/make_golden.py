"""Writes the stored oracle values used by the benchmark's CPU baseline.

Calls only the oracle (and the seeded input generator): for the 4^4 and the
20^3 x 64 CG workloads it records the FP64 CG iteration count to the
workload's tolerance and the oracle's true residual.  Run from the repository
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    'cg_4x4x4x4_m0.05_tol1e-10': dict(dims=(4, 4, 4, 4), eps=0.3, seed=0, mass=0.05, tol=1e-10),
    'cg_20x20x20x64_m0.01_tol1e-8': dict(dims=(20, 20, 20, 64), eps=0.25, seed=0, mass=0.01,
                                         tol=1e-8),
}


def main(names=None):
    out_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'oracle_cg.json')
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    for name, w in WORKLOADS.items():
        if names and name not in names:
            continue
        fat, lng = synth.gauge_field(w['dims'], w['eps'], w['seed'])
        vh = oracle.volume(w['dims']) // 2
        b = synth.gaussian_source(vh, 0)
        t0 = time.time()
        x, it, tr = oracle.cg(w['dims'], fat, lng, w['mass'], b, w['tol'])
        data[name] = dict(w, dims=list(w['dims']), source_seed=0, iterations=it,
                          true_residual=tr, seconds=round(time.time() - t0, 1),
                          note='oracle FP64 CG (textbook, x0 = 0), written by make_golden.py')
        print(name, it, tr)
    with open(out_path, 'w') as fh:
        json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == '__main__':
    main(sys.argv[1:] or None)
