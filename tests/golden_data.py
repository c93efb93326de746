"""Readers for the fixtures in tests/golden/ (numbers the paper prints)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                yield line


def moana_statistics() -> dict:
    """Figure 1 caption: instances, unique quads, instanced quads."""
    return {k: float(v) for k, v in _rows("moana_statistics.txt")}


def table1() -> dict:
    """Table 1: component -> [shot, beach, palms, dunes] percent of compute time."""
    return {r[0]: [float(x) for x in r[1:]] for r in _rows("table1_time_breakdown.txt")}
