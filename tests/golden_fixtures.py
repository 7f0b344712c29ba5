"""Reader of the stored amplitudes under tests/golden/ (written by
tests/golden/make_golden.py from the CPU oracle)."""
import dataclasses
import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclasses.dataclass
class Fixture:
    name: str
    n: int
    p: int
    gamma: list
    beta: list
    edges: np.ndarray  # m x 2 int32
    norm: float
    xs: np.ndarray     # count x n uint8
    amps: np.ndarray   # count complex128


def load(path: str) -> Fixture:
    fields, xs, amps = {}, [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            if key == "x":
                xs.append([int(c) for c in rest[0]])
                amps.append(complex(float(rest[1]), float(rest[2])))
            else:
                fields[key] = rest
    edges = np.array([[int(v) for v in e.split("-")] for e in fields["edges"]], dtype=np.int32)
    return Fixture(os.path.basename(path), int(fields["n"][0]), int(fields["p"][0]),
                   [float(v) for v in fields["gamma"]], [float(v) for v in fields["beta"]], edges,
                   float(fields["norm"][0]), np.array(xs, dtype=np.uint8), np.array(amps))


def all_fixtures():
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))]
