"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Only the oracle (oracle/) computes them; the inputs come from the seeded
input module.  Each file starts with '#' lines naming the workload and the
passage of the paper the computation follows, then `key value` lines with
values printed to 17 significant digits.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1208_2407_gb300 import workloads as wl  # noqa: E402

# sites sampled from the final state of the 256^2 workload (x, y)
C1_SITES = [(0, 0), (255, 255), (128, 128), (133, 128), (140, 131), (120, 110), (150, 140),
            (101, 128), (160, 128), (128, 96), (128, 160), (170, 150), (90, 90), (200, 30),
            (31, 200), (255, 0)]


def c1_values():
    """Config 1: 256^2 FP64, V = 0, packet at (128, 128), sigma 16, kx 0.5,
    theta 0.025, dt 0.05, 100 second-order steps."""
    c = wl.plain_fp64_256()
    re, im = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    m = oracle.moments(re, im)
    kin, pot = oracle.energy(re, im, np.zeros_like(re))
    out = [("norm", m[0]), ("x", m[1] / m[0]), ("y", m[2] / m[0]), ("x2", m[3] / m[0]),
           ("y2", m[4] / m[0]), ("e_kin", kin), ("e_pot", pot)]
    for x, y in C1_SITES:
        out.append(("re[%d,%d]" % (x, y), re[y, x]))
        out.append(("im[%d,%d]" % (x, y), im[y, x]))
    return out


def write(path, header, values):
    with open(path, "w") as f:
        for line in header:
            f.write("# %s\n" % line)
        for k, v in values:
            f.write("%s %.17g\n" % (k, v))


def main():
    write(os.path.join(HERE, "c1_plain_fp64_256.txt"),
          ["256x256 FP64, V = 0, Gaussian packet centre (128, 128), sigma 16, kx 0.5, ky 0",
           "theta = 0.025, dt = 0.05, 100 steps of U2 (Sec. 2, Eq. secondorder; the 2-D",
           "five-part splitting of Sec. 2, open boundaries, +i sin theta, half angle)",
           "written by tests/golden/make_golden.py from the FP64 oracle",
           "moments are sum x|psi|^2 / norm etc.; e_kin = -J sum_pairs 2 Re(conj psi_j psi_k)"],
          c1_values())


if __name__ == "__main__":
    main()
