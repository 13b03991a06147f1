"""Write oracle solutions of the seeded small instances as text fixtures.

Calls only the CPU oracle; run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from gen import CONFIGS, make_problem  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    for name in ("tiny", "grid30_n24"):
        p = make_problem(CONFIGS[name])
        out = oracle.kkt_solve(p)
        path = os.path.join(HERE, f"{name}_solution.txt")
        with open(path, "w") as f:
            f.write(f"# oracle solution of K x = r for the seeded '{name}' instance\n")
            f.write(f"# N={p.N} nA={p.nA} nP={p.nP} nC={p.nC}\n")
            f.write("# inertia " + " ".join(str(int(v)) for v in out["inertia"]) + "\n")
            for v in out["x"]:
                f.write(f"{v:.17e}\n")
        print(path)


if __name__ == "__main__":
    main()
