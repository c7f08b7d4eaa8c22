"""Reader for the stored expected values under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """`key value` lines of tests/golden/<name> as a dict of floats."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def sites(values):
    """(x, y) of the sampled sites, in file order."""
    out = []
    for k in values:
        if k.startswith("re["):
            x, y = k[3:-1].split(",")
            out.append((int(x), int(y)))
    return out
