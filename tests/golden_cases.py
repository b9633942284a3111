"""Loader for the hand-worked fixtures under ``tests/golden/``."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_closed_forms(name: str = "closed_forms.txt"):
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "case":
                cur = {}
                cases[rest.strip()] = cur
            elif key == "end":
                cur = None
            elif key == "n":
                cur["n"] = int(rest)
            elif key == "U":
                cur["U"] = np.array([[float(t) for t in row.split()] for row in rest.split("|")])
            else:
                cur[key] = np.array([float(t) for t in rest.split()])
    return cases
