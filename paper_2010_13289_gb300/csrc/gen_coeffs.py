"""Generate csrc/teno_coeffs.cuh: exact TENO constants for the CUDA kernels.

Derivation (Section 2, Eqs. definitionEq and approximatepolynomial; Section 2.2):
for a stencil of cells j0..j0+r-1 around cell i (Delta x = 1, cell i centred at 0),
the primitive P(x) = int_{j0-1/2}^{x} h takes the values S_q = sum_{m<j0+q} f_m at the
cell edges e_q = j0 - 1/2 + q (q = 0..r).  P is the degree-r Lagrange interpolant of
those r+1 points and the candidate polynomial is h = P'.  Hence
  * the candidate flux h(1/2) = sum_m f_m phi_m(1/2) with phi_m = sum_{q > m-j0} l_q',
  * beta = sum_{j=1}^{r-1} int_{-1/2}^{1/2} (h^(j))^2 dx is a quadratic form in f that
    annihilates constants; written in the differences D_t = f_{j0+t+1} - f_{j0+t}
    (t = 0..r-2) it is D^T Q D with Q symmetric positive definite, emitted as the
    sum of squares sum_t w_t (D_t + sum_{u>t} L_{ut} D_u)^2 (LDL^T factorisation),
  * the optimal weights d_k solve sum_k d_k c_k = c_full (maximal order).
All arithmetic is exact (fractions.Fraction); each constant is written as the
correctly rounded double.  Run:  python paper_2010_13289_gb300/csrc/gen_coeffs.py
"""
import os
from fractions import Fraction as Fr

# candidate stencils S_0..S_5 (incremental width, Fig. incremental_stencil)
CAND = [(-1, 3), (0, 3), (-2, 3), (0, 4), (-3, 4), (0, 5)]  # (j0, r)
FULL = {6: (-2, 6), 8: (-3, 8)}


def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pscale(a, s):
    return [x * s for x in a]


def pder(a):
    return [a[i] * i for i in range(1, len(a))] or [Fr(0)]


def pint_def(a, lo, hi):
    tot = Fr(0)
    for i, c in enumerate(a):
        tot += c * (hi ** (i + 1) - lo ** (i + 1)) / (i + 1)
    return tot


def peval(a, x):
    tot = Fr(0)
    for c in reversed(a):
        tot = tot * x + c
    return tot


def lagrange(nodes, q):
    p = [Fr(1)]
    for j, xj in enumerate(nodes):
        if j != q:
            p = pmul(p, [-xj / (nodes[q] - xj), Fr(1) / (nodes[q] - xj)])
    return p


def basis(j0, r):
    """phi_m(x), m = 0..r-1 (cell j0+m): h(x) = sum_m f_m phi_m(x)."""
    edges = [Fr(2 * j0 - 1, 2) + q for q in range(r + 1)]
    dl = [pder(lagrange(edges, q)) for q in range(r + 1)]
    phis = []
    for m in range(r):
        p = [Fr(0)]
        for q in range(m + 1, r + 1):
            p = padd(p, dl[q])
        phis.append(p)
    return phis


def face_coeffs(j0, r):
    return [peval(p, Fr(1, 2)) for p in basis(j0, r)]


def beta_ldl(j0, r):
    phis = basis(j0, r)
    h = Fr(1, 2)
    Q = [[Fr(0)] * r for _ in range(r)]
    ders = []
    for p in phis:
        ds, cur = [], p
        for _ in range(1, r):
            cur = pder(cur)
            ds.append(cur)
        ders.append(ds)
    for a in range(r):
        for b in range(r):
            Q[a][b] = sum(pint_def(pmul(ders[a][j], ders[b][j]), -h, h) for j in range(r - 1))
    # f_m = f_0 + sum_{t<m} D_t  ->  Qd = T^T Q T, T[m][t] = 1 if t < m
    n = r - 1
    Qd = [[sum(Q[a][b] for a in range(t + 1, r) for b in range(u + 1, r)) for u in range(n)] for t in range(n)]
    # LDL^T
    L = [[Fr(0)] * n for _ in range(n)]
    w = [Fr(0)] * n
    for j in range(n):
        w[j] = Qd[j][j] - sum(L[j][k] ** 2 * w[k] for k in range(j))
        L[j][j] = Fr(1)
        for i in range(j + 1, n):
            L[i][j] = (Qd[i][j] - sum(L[i][k] * L[j][k] * w[k] for k in range(j))) / w[j]
    assert all(x > 0 for x in w)
    return w, L


def solve(A, b):
    """Exact least-squares-free solve of a consistent overdetermined system."""
    m, n = len(A), len(A[0])
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    piv_rows = []
    r = 0
    for c in range(n):
        p = next(i for i in range(r, m) if M[i][c] != 0)
        M[r], M[p] = M[p], M[r]
        for i in range(m):
            if i != r and M[i][c] != 0:
                f = M[i][c] / M[r][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[r])]
        piv_rows.append(r)
        r += 1
    for i in range(r, m):
        assert M[i][n] == 0, "inconsistent"
    return [M[i][n] / M[i][i] for i in range(n)]


def optimal_weights(K):
    j0f, rf = FULL[K]
    cf = face_coeffs(j0f, rf)
    nk = K - 2
    A = [[Fr(0)] * nk for _ in range(rf)]
    for k in range(nk):
        j0, r = CAND[k]
        ck = face_coeffs(j0, r)
        for m in range(r):
            A[j0 + m - j0f][k] = ck[m]
    return solve(A, cf)


def lit(x):
    return repr(float(x))


def main():
    out = ["/* Generated by paper_2010_13289_gb300/csrc/gen_coeffs.py (exact rationals). Do not edit. */",
           "#pragma once", "", "namespace tenom {", ""]
    # candidates: functions of v[] where v[c] = f_i, i.e. f_{i+m} = v[c+m]
    out.append("/* Candidate fluxes f_{k,i+1/2} (Table 1), c = index of f_i in v. */")
    for k, (j0, r) in enumerate(CAND):
        cs = face_coeffs(j0, r)
        terms = " + ".join("(%s) * v[c + %d]" % (lit(cs[m]), j0 + m) for m in range(r))
        out.append("template <int c> __device__ __forceinline__ double cand%d(const double* v) { return %s; }"
                   % (k, terms))
    out.append("")
    out.append("/* Smoothness indicators as sums of squares of difference combinations;")
    out.append("   D[t] = v[t+1] - v[t], e = index in D of the stencil's first difference.  With ABS the")
    out.append("   coefficients are replaced by their magnitudes (evaluated on |D| this bounds the")
    out.append("   rounding error of the form).  T: double, or float for the certified cutoff filter. */")
    names = [("beta%d" % k, j0, r) for k, (j0, r) in enumerate(CAND)] + \
            [("betaK%d" % K, FULL[K][0], FULL[K][1]) for K in (6, 8)]
    for name, j0, r in names:
        w, L = beta_ldl(j0, r)
        n = r - 1
        body = []
        for t in range(n):
            terms = ["D[e + %d]" % t]
            for u in range(t + 1, n):
                if L[u][t] != 0:
                    terms.append("T(ABS ? %s : %s) * D[e + %d]" % (lit(abs(L[u][t])), lit(L[u][t]), u))
            body.append("  const T t%d = %s;" % (t, " + ".join(terms)))
        acc = " + ".join("T(%s) * (t%d * t%d)" % (lit(w[t]), t, t) for t in range(n))
        out.append("/* %s: cells i%+d..i%+d (ABS: the same form with |coefficients|, for error bounds) */"
                   % (name, j0, j0 + r - 1))
        out.append("template <int e, bool ABS = false, class T = double>")
        out.append("__device__ __forceinline__ T %s(const T* D) {" % name)
        out.extend(body)
        out.append("  return %s;" % acc)
        out.append("}")
    out.append("")
    out.append("/* K-point central reconstruction sum_k d_k f_k (all candidates smooth), c = index of f_i */")
    for K in (6, 8):
        j0, r = FULL[K]
        cs = face_coeffs(j0, r)
        terms = " + ".join("(%s) * v[c + %d]" % (lit(cs[m]), j0 + m) for m in range(r))
        out.append("template <int c> __device__ __forceinline__ double central%d(const double* v) { return %s; }"
                   % (K, terms))
    out.append("")
    for K in (6, 8):
        d = optimal_weights(K)
        out.append("/* maximal-order optimal weights d_k, K = %d */" % K)
        out.append("__device__ __forceinline__ double dopt%d(int k) {" % K)
        out.append("  switch (k) {")
        for k, x in enumerate(d):
            out.append("    case %d: return %s;  /* %s */" % (k, lit(x), x))
        out.append("    default: return 0.0;")
        out.append("  }")
        out.append("}")
    out.append("")
    out.append("}  // namespace tenom")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "teno_coeffs.cuh")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
