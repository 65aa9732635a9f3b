"""Write the stored oracle trajectories under tests/golden/ (calls only oracle/)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    c = workloads.PRED_SMALL
    w = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pred_small_trajectory.txt")
    with open(path, "w") as f:
        f.write("# predation 40x40, 100 sheep / 25 wolves, cap 2048/1024, seed 0 (oracle)\n")
        f.write("# step  sheep_after  wolves_after\n")
        for t, st in enumerate(w.step(c["steps"])):
            f.write(f"{t} {st['n_end'][0]} {st['n_end'][1]}\n")


if __name__ == "__main__":
    main()
