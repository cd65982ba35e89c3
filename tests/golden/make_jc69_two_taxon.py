"""Writes jc69_two_taxon.txt: the closed-form likelihood of one site on a
two-taxon tree under JC69 (Jukes and Cantor 1969; the paper's Eq. 1 with the
JC69 generator), and its derivative in the total length T = t_1 + t_2:

  P_same(T) = 1/4 + 3/4 e^{-4T/3},  P_diff(T) = 1/4 - 1/4 e^{-4T/3},
  L_same = pi P_same = (1/4) P_same,  L_diff = (1/4) P_diff,
  dL_same/dT = -(1/4) e^{-4T/3},      dL_diff/dT = (1/12) e^{-4T/3}.

Only the formulas above are used (no library code)."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    rows = []
    for T in (0.0, 1e-4, 0.002, 0.05, 0.3, 1.0, 2.5, 10.0):
        e = math.exp(-4.0 * T / 3.0)
        rows.append((T, 0.25 * (0.25 + 0.75 * e), -0.25 * e,
                     0.25 * (0.25 - 0.25 * e), e / 12.0))
    with open(os.path.join(HERE, "jc69_two_taxon.txt"), "w") as f:
        f.write("# JC69, two taxa, one site: T L_same dL_same/dT L_diff dL_diff/dT\n")
        f.write("# closed form (Jukes and Cantor 1969; Eq. 1 with the JC69 generator);\n")
        f.write("# written by make_jc69_two_taxon.py\n")
        for r in rows:
            f.write(" ".join(repr(x) for x in r) + "\n")


if __name__ == "__main__":
    main()
