"""Writes tests/golden/plan_units_<config>.json: the algorithmic work of
blocking under a given execution plan, counted exactly by the oracle's plan
replay over every candidate pair of the benchmark's full-size relation (units
per class: equality compares, owner-check compares, |a-b| tests, edit-distance
and Jaccard work; see oracle.plan_units).  Only the oracle and the seeded input
generator run here.

  python tests/golden/make_plan_units.py c2 "<program>"

<program> lists the plan's distinct non-equality predicates in execution
order as indices into oracle.distinct_predicates(mds) (comma separated), the
numbering hb_plan reports in hb_plan_info.op_pred.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main(config, program_ids):
    if config != "c2":
        raise SystemExit("only the single-table benchmark workload (c2) is counted")
    t, mds = synth.config2()
    dp = oracle.distinct_predicates(mds)
    program = [dp[i] for i in program_ids]
    t0 = time.time()
    units = oracle.plan_units(t, mds, program)
    d = {"config": config, "program_ids": program_ids, "program": [list(p) for p in program], "units": units,
         "seconds": round(time.time() - t0, 1),
         "command": f"python tests/golden/make_plan_units.py {config} \"{','.join(map(str, program_ids))}\""}
    with open(os.path.join(HERE, f"plan_units_{config}.json"), "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(json.dumps(d), flush=True)


if __name__ == "__main__":
    main(sys.argv[1], [int(x) for x in sys.argv[2].split(",")])
