"""Writes vzero_hbar.txt: the discrete effective Hamiltonian for V = 0.

With V = 0 and constant data every candidate of a line is const + k_a[d], so a
step adds min_d k_a[d] along each axis and the discrete constant of
Prop. prop:klm is  -sum_a min_d k_a[d] / h,  k_a[d] = h (v^2/2 - P_a v),
v = d dx_a / h  (eq. cost2 with the Lagrangian of Sec. 2.1).  Evaluated here
in exact rational arithmetic from the binary64 parameters of each workload; no
code of the scheme is used.
"""
import os
from fractions import Fraction
from math import floor

WORKLOADS = {  # name: (dx per axis, h, P per axis)
    "line256": ((1 / 256,), 0.05, (0.3,)),
    "grid1024": ((1 / 1024,) * 2, 0.02, (0.3, 0.1)),
    "cube256": ((1 / 256,) * 3, 0.02, (0.2, -0.1, 0.35)),
    "adjoint512": ((1 / 512,) * 2, 0.02, (0.3, 0.1)),
}


def kmin(dx, h, P):
    dx, h, P = Fraction(dx), Fraction(h), Fraction(P)
    ds = floor(P * h / dx)
    vals = []
    for d in range(ds - 3, ds + 5):
        v = d * dx / h
        vals.append(h * (v * v / 2 - P * v))
    return min(vals)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vzero_hbar.txt")
    with open(out, "w") as f:
        f.write("# discrete effective Hamiltonian for V = 0 (Prop. prop:klm, eq. cost2),\n")
        f.write("# exact rationals rounded to binary64; written by make_vzero_hbar.py\n")
        for name, (dx, h, P) in WORKLOADS.items():
            hb = -sum(kmin(dx[a], h, P[a]) for a in range(len(P))) / Fraction(h)
            f.write("%s %.17g\n" % (name, float(hb)))


if __name__ == "__main__":
    main()
