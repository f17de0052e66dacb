"""Reader for the small text fixtures under tests/golden/."""
import math
import os
from fractions import Fraction

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok):
    env = {"sqrt": math.sqrt}
    try:
        return float(Fraction(tok))
    except ValueError:
        return float(eval(tok, {"__builtins__": {}}, env))


def read(name):
    """Return a list of (fields...) tuples with numeric tokens converted to float."""
    rows = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def values(tokens):
    return [_num(t) for t in tokens]
