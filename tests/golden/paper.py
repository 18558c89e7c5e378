"""Reader for the paper's printed numbers in paper_numbers.txt."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def paper_numbers() -> dict:
    out = {}
    with open(os.path.join(_HERE, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            out[key] = float(val)
    return out
