"""Reader of the thesis's tables transcribed under tests/golden/."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    """Rows of numbers of a golden file (comment lines dropped)."""
    out = []
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append([float(v) for v in line.split()])
    return out


def rel_error(name, W, column=-1):
    """The relative H^1 error of degree W as a fraction (the tables print %)."""
    for r in rows(name):
        if int(r[0]) == W:
            return r[column] / 100.0
    raise KeyError((name, W))
