"""Writes the closed-form fixtures of tests/golden/ without touching the
oracle.  Each value is a textbook closed form, derived in the comments.

  python tests/golden/make_golden.py
"""
import math
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def fd_weights_by_vandermonde(M):
    """Centred second-derivative weights of order 2M from the moment
    conditions sum_k w_k k^{2m} = 2 delta_{m,1}, m = 0..M, solved exactly in
    rationals (the symmetric stencil w_{-k} = w_k)."""
    n = M + 1
    # unknowns c_0 = w_0, c_k = 2 w_k (k >= 1): sum_k c_k k^{2m} = 2 delta_{m1}
    A = [[Fraction(k) ** (2 * m) if not (k == 0 and m == 0) else Fraction(1) for k in range(n)]
         for m in range(n)]
    for m in range(1, n):
        A[m][0] = Fraction(0)
    b = [Fraction(2) if m == 1 else Fraction(0) for m in range(n)]
    # Gauss-Jordan elimination in exact arithmetic
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                b[r] -= f * b[col]
    c = [b[i] / A[i][i] for i in range(n)]
    return [c[0]] + [ck / 2 for ck in c[1:]]


def main():
    w = fd_weights_by_vandermonde(6)
    with open(os.path.join(HERE, "fd12_weights.txt"), "w") as f:
        f.write("# 12th-order centred second-derivative weights w_0..w_6 (rational),\n")
        f.write("# from the moment conditions of a symmetric 13-point stencil solved in\n")
        f.write("# exact arithmetic (make_golden.py).  Sec. II.A: high-order centred FD.\n")
        for k, x in enumerate(w):
            f.write("%d %d %d\n" % (k, x.numerator, x.denominator))
    # Normalised Gaussian density rho = (2 pi s^2)^{-3/2} exp(-r^2 / 2 s^2):
    #   Hartree self-energy U = (1/2) int rho V = 1/(2 sqrt(pi) s)
    #   (V = erf(r / (sqrt(2) s)) / r; the integral is the classic
    #   self-energy of a Gaussian charge cloud);
    #   Slater exchange of the fully polarised density,
    #   E_x = -(3/4)(6/pi)^{1/3} int rho^{4/3}, with
    #   int rho^{4/3} = (2 pi s^2)^{-2} (3 pi s^2 / 2)^{3/2}.
    with open(os.path.join(HERE, "gaussian_closed_forms.txt"), "w") as f:
        f.write("# sigma  U_hartree  E_x_polarised  (closed forms; see make_golden.py)\n")
        for s in (0.5, 0.75, 1.0):
            U = 1.0 / (2.0 * math.sqrt(math.pi) * s)
            I43 = (2 * math.pi * s * s) ** -2 * (1.5 * math.pi * s * s) ** 1.5
            Ex = -0.75 * (6.0 / math.pi) ** (1.0 / 3.0) * I43
            f.write("%.2f %.15e %.15e\n" % (s, U, Ex))


if __name__ == "__main__":
    main()
