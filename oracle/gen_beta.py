"""Generate oracle/beta_forms.h: the exact rational data the oracle needs for the
TENO smoothness indicators (Section 2.2, the beta_{k,r} definition under the
scale-separation equation) and for the candidate polynomials (Section 2, Eqs.
definitionEq and approximatepolynomial).

Test infrastructure only (part of the CPU oracle).  Run:  python oracle/gen_beta.py

For a stencil of cells m = j0..j1 (offsets from cell i, Delta x = 1, cell i
centred at x = 0) the candidate polynomial h_k(x) = sum_l a_l x^l is the one whose
cell averages over the stencil cells equal the point values f_m
(Eq. definitionEq with Eq. approximatepolynomial).  Writing a = M f, the paper's
indicator is

    beta = sum_{j=1}^{r-1} int_{-1/2}^{1/2} (d^j h / dx^j)^2 dx   (Delta x = 1)
         = sum_{l,l'>=1} G[l][l'] a_l a_l'

with G[l][l'] = sum_j int (d^j x^l)(d^j x^l') dx.  Rows l >= 1 of M sum to zero
(derivatives ignore constants), so the oracle evaluates a_l = sum_m M[l][m](f_m - f_i),
which is the same number in exact arithmetic and avoids cancelling a large mean.

Emitted:  M rows l = 1..r-1 (r columns) and G (r-1 x r-1) for the candidate stencils
S_0..S_5 (Fig. incremental_stencil / Table 1) and for the K-point full stencils
(K = 6: i-2..i+3, K = 8: i-3..i+4), plus h_k(1/2) coefficients (which must equal
Table 1; checked by the tests, not used by the oracle).
"""
import os
import sympy as sp

X = sp.Symbol("x")

# stencil cell offsets relative to i (Fig. incremental_stencil, Table 1 columns)
STENCILS = {
    "S0": [-1, 0, 1],
    "S1": [0, 1, 2],
    "S2": [-2, -1, 0],
    "S3": [0, 1, 2, 3],
    "S4": [-3, -2, -1, 0],
    "S5": [0, 1, 2, 3, 4],
    "F6": [-2, -1, 0, 1, 2, 3],
    "F8": [-3, -2, -1, 0, 1, 2, 3, 4],
}


def forms(offsets):
    r = len(offsets)
    h = sp.Rational(1, 2)
    # A[m][l] = int_{m-1/2}^{m+1/2} x^l dx  (cell average of the monomial, Eq. definitionEq)
    A = sp.Matrix(r, r, lambda mi, l: sp.integrate(X**l, (X, offsets[mi] - h, offsets[mi] + h)))
    M = A.inv()  # a = M f
    G = sp.zeros(r - 1, r - 1)
    for l in range(1, r):
        for lp in range(1, r):
            s = 0
            for j in range(1, r):
                s += sp.integrate(sp.diff(X**l, X, j) * sp.diff(X**lp, X, j), (X, -h, h))
            G[l - 1, lp - 1] = sp.nsimplify(s)
    face = [sp.nsimplify(sum(M[l, mi] * h**l for l in range(r))) for mi in range(r)]
    return M, G, face


def rat(q):
    q = sp.Rational(q)
    if q.q == 1:
        return "%d.0" % q.p
    return "(%d.0/%d.0)" % (q.p, q.q)


def main():
    out = []
    out.append("/* Generated by oracle/gen_beta.py (sympy, exact rationals). Do not edit.\n"
               "   Oracle test infrastructure: see that script's docstring for the definitions. */")
    out.append("#pragma once")
    for name, offs in STENCILS.items():
        M, G, face = forms(offs)
        r = len(offs)
        out.append("/* stencil %s: cells i%+d..i%+d, r = %d */" % (name, offs[0], offs[-1], r))
        out.append("static const int ORC_%s_R = %d;" % (name, r))
        out.append("static const int ORC_%s_J0 = %d;" % (name, offs[0]))
        rows = []
        for l in range(1, r):
            rows.append("{" + ", ".join(rat(M[l, mi]) for mi in range(r)) + "}")
        out.append("static const double ORC_%s_M[%d][%d] = {%s};" % (name, r - 1, r, ",\n    ".join(rows)))
        grows = []
        for a in range(r - 1):
            grows.append("{" + ", ".join(rat(G[a, b]) for b in range(r - 1)) + "}")
        out.append("static const double ORC_%s_G[%d][%d] = {%s};" % (name, r - 1, r - 1, ",\n    ".join(grows)))
        out.append("static const double ORC_%s_FACE[%d] = {%s};" % (name, r, ", ".join(rat(c) for c in face)))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "beta_forms.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
