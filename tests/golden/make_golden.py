"""Write the stored oracle trajectories under tests/golden/ (calls only oracle/)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import hashlib  # noqa: E402

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

STATE_ARRAYS = ("sheep.active", "sheep.cell", "sheep.energy", "sheep.id", "sheep.age",
                "wolf.active", "wolf.cell", "wolf.energy", "wolf.id", "wolf.age", "grass.grown", "grass.wait")


def state_sha256(arrays: dict) -> str:
    """SHA-256 over the canonical state arrays (int32 little-endian, fixed order)."""
    h = hashlib.sha256()
    for k in STATE_ARRAYS:
        h.update(np.ascontiguousarray(arrays[k], dtype="<i4").tobytes())
    return h.hexdigest()


def oracle_state(w) -> dict:
    st = w.state()
    grown = st["grass.grown"]
    st["grass.wait"] = np.where(grown != 0, 0, np.maximum(st["grass.countdown"], 1)).astype(np.int32)
    return st


def large():
    c = workloads.PRED_LARGE
    w = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pred_large_trajectory.txt")
    rows = []
    for t in range(c["steps"]):
        s = w.step()[0]
        rows.append((t, s["n_start"][0], s["n_start"][1], s["parents"][0], s["parents"][1], s["births"][0],
                     s["births"][1], s["starved"][0], s["starved"][1], s["eaten"], s["grass_eaten"],
                     s["n_end"][0], s["n_end"][1], s["hw"][0], s["hw"][1]))
    digest = state_sha256(oracle_state(w))
    with open(path, "w") as f:
        f.write("# predation 2048x2048, 1,000,000 sheep / 250,000 wolves, cap 8Mi/4Mi, seed 1 (oracle)\n")
        f.write(f"# final_state_sha256 {digest}\n")
        f.write("# step n_start_s n_start_w parents_s parents_w births_s births_w starved_s starved_w "
                "eaten grass n_end_s n_end_w hw_s hw_w\n")
        for r in rows:
            f.write(" ".join(str(int(x)) for x in r) + "\n")


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "large":
        large()
        return
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
