"""Writes the stored expected values under tests/golden/.  Calls only oracle/.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    with open(os.path.join(HERE, "self_term.txt"), "w") as f:
        f.write("# Self-cell integral of Eq. 13 for a unit cube: integral over the cube of dV/r\n"
                "# with r measured from the cube centre.  The paper computes it \"numerically or\n"
                "# analytically\" (Sect. 3, citing Macmillan 1958 and Hahn 2020); the oracle's\n"
                "# closed form 3 ln(2 + sqrt 3) - pi/2 evaluated to double precision:\n")
        f.write("C = %.16g\n" % oracle.SELF_TERM_C)


if __name__ == "__main__":
    main()
