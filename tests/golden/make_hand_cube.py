"""Write hand_cube.txt: closed-form residual and gradient on the 8-node cube.

The mesh is the unit cube's 8 corners (id = x + 2y + 4z) joined by its 12
edges, each running from the lower to the upper corner along one axis, with
the unit axis vector as the dual-face normal (area 1).  The state is at rest:
rho = 1, u = 0, c = 0 and p_i = 1 + i/8, so rho E = p / (gamma - 1).

At rest the Euler flux through a face is pure pressure, (0, p n, 0, 0), and
the wave speed of a state is its sound speed a = sqrt(gamma p / rho) (|n| = 1).
The Rusanov flux of edge (i, j) therefore has the closed form
    momentum   (p_i + p_j)/2 * n
    energy     -sqrt(gamma * max(p_i, p_j)) * (p_j - p_i) / (2 (gamma - 1))
and zero mass and scalar components; R_i = sum(+F) over edges leaving i
minus sum(F) over edges entering i.  The unscaled Green-Gauss sums are, per
component k and axis d, +-(q_i,k + q_nbr,k)/2 with + when i is the lower end.

This script evaluates these closed forms in 40-digit decimal arithmetic.  It
imports nothing from the library or the oracle.
"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 40
GAMMA = Decimal("1.4")


def main():
    nodes = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    nid = {p: k for k, p in enumerate(nodes)}
    p = [Decimal(1) + Decimal(i) / Decimal(8) for i in range(8)]
    q = [[Decimal(1), Decimal(0), Decimal(0), Decimal(0),
          p[i] / (GAMMA - 1), Decimal(0)] for i in range(8)]
    R = [[Decimal(0)] * 6 for _ in range(8)]
    G = [[Decimal(0)] * 18 for _ in range(8)]
    for pt in nodes:
        for d in range(3):
            if pt[d] != 0:
                continue
            up = list(pt)
            up[d] = 1
            i, j = nid[pt], nid[tuple(up)]
            F = [Decimal(0)] * 6
            F[1 + d] = (p[i] + p[j]) / 2
            s = (GAMMA * max(p[i], p[j])).sqrt()
            F[4] = -s * (p[j] - p[i]) / (2 * (GAMMA - 1))
            for k in range(6):
                R[i][k] += F[k]
                R[j][k] -= F[k]
                c = (q[i][k] + q[j][k]) / 2
                G[i][3 * k + d] += c
                G[j][3 * k + d] -= c
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "hand_cube.txt")
    with open(out, "w") as fh:
        fh.write("# closed-form first-order residual R (8 x 6) and unscaled "
                 "Green-Gauss sums Graw (8 x 18)\n# on the 8-node unit cube at "
                 "rest, p_i = 1 + i/8; written by make_hand_cube.py\n")
        for i in range(8):
            fh.write("R %d " % i + " ".join("%.25e" % v for v in R[i]) + "\n")
        for i in range(8):
            fh.write("G %d " % i + " ".join("%.25e" % v for v in G[i]) + "\n")


if __name__ == "__main__":
    main()
