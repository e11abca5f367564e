"""Write the stored expected values under tests/golden/ by calling the FP64 oracle only.

    python tests/golden/make_golden.py

Each fixture is plain text: a header of '#' lines (what, how, the paper passage the
workload follows), then one value per line. Inputs come from
paper_1907_13013_gb300.inputs (seeded generators holding no solver arithmetic).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import iterations as it  # noqa: E402
from paper_1907_13013_gb300 import inputs  # noqa: E402


def write(name, header, phi0):
    with open(os.path.join(HERE, name), "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        for v in phi0.ravel():
            f.write("%.17e\n" % v)


def main():
    cases = [
        ("plain_hg_slab", inputs.plain_hg_slab(),
         "1 cm, 200 cells, S16, HG g=0.9 to L=15, sigma_t=101, sigma_s0=100, isotropic Q=1, vacuum"),
        ("precision_srk_slab", inputs.precision_srk_slab(),
         "1 cm, 2000 cells, S64, screened Rutherford eta=1e-5 to L=63, sigma_s0=1000, sigma_a=0.01, Q=1 on z<0.5, vacuum"),
    ]
    for name, p, desc in cases:
        for lap in ("mpd", "wfd"):
            _, n10 = it.fpsa_source_iteration(p, lap, tol=1e-10)
            phi, n13 = it.fpsa_source_iteration(p, lap, tol=1e-13)
            hdr = [
                "scalar flux phi_0 at the LD nodes [cell][node], FP64 oracle, FPSA-SI with %s "
                "(Eqs. predict, correct, iterate; Eq. fp-mpd / w_wfd)" % lap.upper(),
                "workload: " + desc,
                "iterations to relative change 1e-10: %d" % n10,
                "iterations to relative change 1e-13 (values below): %d" % n13,
                "written by tests/golden/make_golden.py (oracle only)",
            ]
            write("%s_fpsa_%s_phi0.txt" % (name, lap), hdr, phi[..., 0])
            print(name, lap, n10, n13)


if __name__ == "__main__":
    main()
