"""Write the number of canonical shell quartets that survive the screening of
the HSE cluster workload (Schwarz 1e-8 and density screening 1e-8 with the
erfc kernel, w = 0.11; P cut at 14 bohr) to tests/golden/, computed by the
oracle alone (oracle.count_quartets): Schwarz bounds of every shell pair and
the survival predicate of every candidate quartet, no integral of a quartet.

    python oracle/count_quartets.py --atoms 400
    python oracle/count_quartets.py --atoms 400 --dddd-above 1e-5

The second form counts only the (dd|dd) quartets whose bound Q_IJ Q_KL P_scr
exceeds the given value (the quartets a mixed build with FP64 promotion
restricted to total l >= 8 routes to FP64): the same predicate with eps set to
that value, on the d shells alone (Schwarz bounds and shell-pair |P| maxima
depend only on the two shells of a pair, so the sub-basis changes neither).

Test infrastructure: the benchmark's reference arm uses the stored count to
express the oracle's quartets/s in builds/s, and tests compare the GPU build's
count with it.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--atoms", type=int, default=400)
    ap.add_argument("--dddd-above", type=float, default=None)
    args = ap.parse_args()
    s, P = synth.config2(args.atoms)
    mask = synth.atom_pair_mask(s, 14.0)
    P = P * synth.expand_atom_mask(s, mask)
    eps, name, what = 1e-8, f"quartet_count_hse_c{args.atoms}.json", ""
    cmd = "python oracle/count_quartets.py --atoms %d" % args.atoms
    if args.dddd_above is not None:
        s, P = synth.shell_subset(s, P, [2])
        eps = args.dddd_above
        name = f"quartet_count_hse_c{args.atoms}_dddd_above{args.dddd_above:g}.json"
        what = f"; (dd|dd) quartets only, with Q_IJ Q_KL P_scr > {args.dddd_above:g}"
        cmd += f" --dddd-above {args.dddd_above:g}"
    t0 = time.time()
    n, _ = oracle.count_quartets(oracle.Basis(s), P, kernel=oracle.KERNEL_ERFC, omega=0.11, tau=1e-8,
                                 density_screen=True, eps=eps)
    out = {"workload": f"{args.atoms}-atom C/H cluster (synth.config2), HSE erfc w=0.11, Schwarz 1e-8 + density "
                       f"screening 1e-8, P cut 14 bohr" + what,
           "canonical_quartets": n, "written_by": cmd,
           "oracle_seconds": round(time.time() - t0, 1), "threads": oracle.max_threads()}
    path = os.path.join(ROOT, "tests", "golden", name)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
