"""Pins of the oracle's scalar TENO-M reconstruction (Sections 2-3) against what the
paper prints and what mathematics fixes.  CPU only."""
import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from conftest import read_golden


def table1():
    rows = {}
    for r in read_golden("table1.txt"):
        k = int(r[0])
        trip = [int(x) for x in r[1:]]
        rows[k] = {trip[j]: trip[j + 1] / trip[j + 2] for j in range(0, len(trip), 3)}
    return rows


def seq_from(fun, K, i0=0.0, h=1.0):
    """Values f_m, m = i-K/2+1 .. i+K/2, of fun at x_m = i0 + m h (i at m = 0)."""
    ms = np.arange(-K // 2 + 1, K // 2 + 1)
    return fun(i0 + ms * h), ms


def cell_avg_poly(coef, m):
    """Average over [m-1/2, m+1/2] of the polynomial with coefficients coef (x-centred)."""
    ic = P.polyint(coef)
    return P.polyval(m + 0.5, ic) - P.polyval(m - 0.5, ic)


@pytest.mark.parametrize("K", [6, 8])
def test_candidates_equal_table1(orc, K):
    """The oracle's candidate fluxes are Table 1 applied to the stencil values."""
    S = orc.make_scheme(K)
    t1 = table1()
    rng = np.random.default_rng(11)
    for _ in range(20):
        f = rng.normal(size=K)
        parts = orc.recon_parts(S, f)
        for k in range(K - 2):
            want = sum(c * f[m + K // 2 - 1] for m, c in t1[k].items())
            assert parts["cand"][k] == pytest.approx(want, rel=1e-14, abs=1e-14)


def test_table1_is_primitive_reconstruction():
    """Each Table 1 row reproduces h(x_{i+1/2}) exactly when the f_m are cell averages of
    a polynomial h of degree < r_k (Eqs. definitionEq, approximatepolynomial)."""
    t1 = table1()
    rng = np.random.default_rng(3)
    for k, row in t1.items():
        r = len(row)
        for _ in range(5):
            coef = rng.normal(size=r)
            got = sum(c * cell_avg_poly(coef, m) for m, c in row.items())
            assert got == pytest.approx(P.polyval(0.5, coef), rel=1e-12, abs=1e-12)


def test_generator_face_rows_match_table1():
    """The oracle's own beta-form generator derives the same face coefficients."""
    sp = pytest.importorskip("sympy")
    import oracle.gen_beta as G
    t1 = table1()
    for k in range(6):
        offs = G.STENCILS["S%d" % k]
        _, _, face = G.forms(offs)
        for mi, m in enumerate(offs):
            assert float(face[mi]) == pytest.approx(t1[k][m], rel=1e-15)


@pytest.mark.parametrize("K", [6, 8])
def test_optimal_weights_give_central_scheme(orc, K):
    """Reading: maximal-order d_k.  sum_k d_k f_k must be exact for polynomials of degree
    K-1 (order K) and equal the K-point central reconstruction."""
    d = orc.default_weights(K)
    assert d.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(d > 0)
    S = orc.make_scheme(K)
    rng = np.random.default_rng(5)
    for _ in range(5):
        coef = rng.normal(size=K)
        ms = np.arange(-K // 2 + 1, K // 2 + 1)
        f = np.array([cell_avg_poly(coef, m) for m in ms])
        parts = orc.recon_parts(S, f)
        lin = float(np.dot(d, parts["cand"]))
        assert lin == pytest.approx(P.polyval(0.5, coef), rel=1e-11, abs=1e-11)
    # degree K is not reproduced (the order is exactly K)
    coef = np.zeros(K + 1)
    coef[K] = 1.0
    ms = np.arange(-K // 2 + 1, K // 2 + 1)
    f = np.array([cell_avg_poly(coef, m) for m in ms])
    lin = float(np.dot(d, orc.recon_parts(S, f)["cand"]))
    assert abs(lin - P.polyval(0.5, coef)) > 1e-6


def jiang_shu(f):
    """Textbook Jiang-Shu indicators of the three 3-point stencils (f = f_{i-2}..f_{i+2})."""
    fm2, fm1, f0, fp1, fp2 = f
    b0 = 0.25 * (fm1 - fp1) ** 2 + 13 / 12 * (fm1 - 2 * f0 + fp1) ** 2
    b1 = 0.25 * (3 * f0 - 4 * fp1 + fp2) ** 2 + 13 / 12 * (f0 - 2 * fp1 + fp2) ** 2
    b2 = 0.25 * (fm2 - 4 * fm1 + 3 * f0) ** 2 + 13 / 12 * (fm2 - 2 * fm1 + f0) ** 2
    return b0, b1, b2


@pytest.mark.parametrize("K", [6, 8])
def test_beta_r3_equals_jiang_shu(orc, K):
    S = orc.make_scheme(K)
    rng = np.random.default_rng(7)
    for _ in range(50):
        f = rng.normal(size=K)
        parts = orc.recon_parts(S, f)
        c = K // 2 - 1  # index of f_i
        js = jiang_shu(f[c - 2:c + 3])
        for k in range(3):
            assert parts["beta"][k] == pytest.approx(js[k], rel=1e-13)


def beta_exact(coef):
    """sum_{j>=1} int_{-1/2}^{1/2} (h^(j))^2 dx for polynomial h (Delta x = 1)."""
    tot = 0.0
    c = np.array(coef, dtype=float)
    while True:
        c = P.polyder(c)
        if c.size == 0 or not np.any(c):
            break
        sq = P.polymul(c, c)
        isq = P.polyint(sq)
        tot += P.polyval(0.5, isq) - P.polyval(-0.5, isq)
    return tot


STENCIL_OFFS = {0: (-1, 1), 1: (0, 2), 2: (-2, 0), 3: (0, 3), 4: (-3, 0), 5: (0, 4)}


@pytest.mark.parametrize("K", [6, 8])
def test_beta_definition_on_exact_polynomials(orc, K):
    """When the f_m are cell averages of a polynomial h of degree < r_k, the candidate
    polynomial is h itself, so beta_{k,r} is the integral of Eq. measureTENO (2nd) of h;
    likewise beta_K for degree < K."""
    S = orc.make_scheme(K)
    rng = np.random.default_rng(13)
    ms = np.arange(-K // 2 + 1, K // 2 + 1)
    for k in range(K - 2):
        lo, hi = STENCIL_OFFS[k]
        r = hi - lo + 1
        for _ in range(3):
            coef = rng.normal(size=r)
            f = np.array([cell_avg_poly(coef, m) for m in ms])
            got = orc.recon_parts(S, f)["beta"][k]
            assert got == pytest.approx(beta_exact(coef), rel=1e-10)
    coef = rng.normal(size=K)
    f = np.array([cell_avg_poly(coef, m) for m in ms])
    assert orc.recon_parts(S, f)["betaK"] == pytest.approx(beta_exact(coef), rel=1e-10)


@pytest.mark.parametrize("K", [6, 8])
def test_beta_invariances(orc, K):
    S = orc.make_scheme(K)
    rng = np.random.default_rng(17)
    f = rng.normal(size=K)
    p0 = orc.recon_parts(S, f)
    p1 = orc.recon_parts(S, f + 123.0)
    p2 = orc.recon_parts(S, 3.0 * f)
    np.testing.assert_allclose(p1["beta"], p0["beta"], rtol=1e-10)
    np.testing.assert_allclose(p2["beta"], 9 * p0["beta"], rtol=1e-13)
    assert p2["betaK"] == pytest.approx(9 * p0["betaK"], rel=1e-13)
    pc = orc.recon_parts(S, np.full(K, 2.5))
    assert np.all(pc["beta"] == 0) and pc["betaK"] == 0


@pytest.mark.parametrize("K", [6, 8])
def test_tau_is_sixth_order(orc, K):
    """Eq. taukTENO: tau_K = O(dx^6) on smooth data (ratio ~64 per halving)."""
    S = orc.make_scheme(K)
    taus = []
    for h in [0.1, 0.05, 0.025]:
        f, _ = seq_from(lambda x: np.sin(x) + 0.3 * np.cos(2 * x), K, i0=0.4, h=h)
        taus.append(orc.recon_parts(S, f)["tau"])
    r1, r2 = taus[0] / taus[1], taus[1] / taus[2]
    assert 45 < r1 < 90 and 45 < r2 < 90, (r1, r2)


@pytest.mark.parametrize("K", [6, 8])
def test_linear_reproduction_on_smooth_data(orc, K):
    """Smooth data: all delta_k = 1 and TENO-M equals the central linear scheme
    (Section 3.3: w_k = d_k without renormalisation)."""
    S = orc.make_scheme(K)
    rows = []
    for x0 in np.linspace(0, 6, 40):
        f, _ = seq_from(lambda x: np.sin(x) + 2.0, K, i0=x0, h=0.05)
        rows.append(f)
    v = np.array(rows)
    fh, bits, _, _, _ = orc.recon(S, v)
    assert np.all(bits == (1 << (K - 2)) - 1)
    central = {6: np.array([1, -8, 37, 37, -8, 1]) / 60.0,
               8: np.array([-3, 29, -139, 533, 533, -139, 29, -3]) / 840.0}[K]
    np.testing.assert_allclose(fh, v @ central, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("K,lim", [(6, 0), (8, 0), (6, 1), (8, 1)])
def test_discontinuity_marks_nonsmooth(orc, K, lim):
    """A step inside the stencil marks the candidates that cross it nonsmooth, and the
    result stays within the data range (no overshoot at a step)."""
    S = orc.make_scheme(K, limiter=lim)
    ms = np.arange(-K // 2 + 1, K // 2 + 1)
    f = np.where(ms <= 1, 1.0, 0.0)   # jump between i+1 and i+2
    fh, bits, _, _, _ = orc.recon(S, f[None, :])
    assert bits[0] & 1  # S0 = {i-1, i, i+1} is smooth
    assert not (bits[0] >> 1) & 1  # S1 = {i, i+1, i+2} crosses the jump
    assert -1e-12 <= fh[0] <= 1.0 + 1e-12


@pytest.mark.parametrize("K", [6, 8])
@pytest.mark.parametrize("a,b,J", [(1.0, 1.0, 100.0), (-3.0, 0.25, -50.0), (10.0, -2.0, 1e3)])
def test_renormalised_weights_reproduce_the_smooth_side(orc, K, a, b, J):
    """Classical TENO weights (Eq. weight_renormalize): linear data a + b m with a jump J
    between i+1 and i+2.  Exactly the candidates upwind of the jump (S0, S2 and, for K = 8,
    S4) are smooth; each reproduces linear data exactly, so the renormalised combination
    sum_{smooth} d_k f_k / sum_{smooth} d_k is the linear value at x_{i+1/2}, a + b/2,
    whatever the jump (a dropped denominator or a wrong candidate set misses it)."""
    S = orc.make_scheme(K, weights=orc.W_TENO)
    ms = np.arange(-K // 2 + 1, K // 2 + 1)
    v = a + b * ms + np.where(ms >= 2, J, 0.0)
    fh, bits, _, _, _ = orc.recon(S, v[None, :])
    smooth = (1 << 0) | (1 << 2) | ((1 << 4) if K == 8 else 0)
    assert bits[0] == smooth
    assert abs(fh[0] - (a + 0.5 * b)) <= 1e-13 * (abs(a) + abs(b))


def test_cutoff_tie_is_smooth(orc):
    """Eq. cut-off: delta_k = 0 only for chi_k < C_T; with C_T = 0 every stencil is
    smooth, with C_T = 2 every stencil is nonsmooth (chi_k <= 1)."""
    rng = np.random.default_rng(23)
    v = rng.normal(size=(30, 6))
    _, b0, _, _, _ = orc.recon(orc.make_scheme(6, ct_const=0.0), v)
    _, b1, _, _, _ = orc.recon(orc.make_scheme(6, ct_const=2.0), v)
    assert np.all(b0 == 15) and np.all(b1 == 0)


def minmod2(x, y):
    return 0.5 * (np.sign(x) + np.sign(y)) * min(abs(x), abs(y))


def test_mp_bounds_contain_fi_and_median_identity(orc):
    """Section 3.2.2: both intervals of Eq. value_min_max contain f_i, so
    f^{L,min} <= f_i <= f^{L,max}, and the median is the identity inside the bounds."""
    S = orc.make_scheme(6, ct_const=2.0)  # forces delta_k = 0 for every k
    rng = np.random.default_rng(29)
    for _ in range(200):
        f = rng.normal(size=6)
        p = orc.recon_parts(S, f)
        fi = f[2]
        assert p["mpmin"] <= fi <= p["mpmax"]
        fh, bits, _, _, _ = orc.recon(S, f[None, :])
        assert bits[0] == 0
        cl = [min(max(c, p["mpmin"]), p["mpmax"]) for c in p["cand"]]
        assert fh[0] == pytest.approx(float(np.dot(orc.default_weights(6), cl)), rel=1e-13, abs=1e-13)


def test_mp_bounds_textbook_example(orc):
    """Suresh-Huynh bounds on a hand-worked sequence (Eqs. curvature to value_min_max).
    f = (0, 0, 1, 3, 4, 4): d_{i-1} = 1, d_i = 1, d_{i+1} = -1, d^{M4}_{i+1/2} = 0,
    d^{M4}_{i-1/2} = 1; f^{UL} = 1 + 1.25 = 2.25, f^{MD} = 2, f^{LC} = 1.5 + 4/3;
    f^{L,min} = max(min(1, 3, 2), min(1, 2.25, 2.8333)) = 1,
    f^{L,max} = min(max(1, 3, 2), max(1, 2.25, 2.8333)) = 2.8333."""
    S = orc.make_scheme(6)
    p = orc.recon_parts(S, np.array([0.0, 0.0, 1.0, 3.0, 4.0, 4.0]))
    assert p["mpmin"] == pytest.approx(1.0, abs=1e-15)
    assert p["mpmax"] == pytest.approx(1.5 + 4.0 / 3.0, rel=1e-15)


def tvd5_paper(f):
    """Eqs. high order TVD, TVDhighorder2, TVDbeta exactly as printed (needs nonzero
    differences); f = f_{i-2}..f_{i+2}."""
    fm2, fm1, f0, fp1, fp2 = f
    dm = f0 - fm1
    dp = fp1 - f0
    r_j = dp / dm
    r_jm1 = (f0 - fm1) / (fm1 - fm2)
    r_jp1 = (fp2 - fp1) / (fp1 - f0)
    beta = (-2.0 / r_jm1 + 11.0 + 24.0 * r_j - 3.0 * r_j * r_jp1) / 30.0
    phi = max(0.0, min(2.0, 2.0 * r_j, beta))
    return f0 + 0.5 * phi * dm


@pytest.mark.parametrize("curv,beta,fmax", [("M4", 4.0, 2.25), ("MM", 4.0, 1.5 + 4.0 / 3.0),
                                             ("MM", 3.0, 2.5), ("MM", 1.0, 2.25)])
def test_mp_bounds_curvature_variants_worked_example(orc, curv, beta, fmax):
    """Hand-worked sequence f = (0, 0, 1, 10, 27, 27) for the curvature variants of
    Section 4 (d^{MM}_{i+1/2} = minmod(d_i, d_{i+1})) and beta of Eq. large_curvature:
    d_{i-1} = 1, d_i = 8, d_{i+1} = 8; d_{i+1/2} = 8 under both measures, d_{i-1/2} =
    minmod4(-4, 31, 1, 8) = 0 under M4 but minmod(1, 8) = 1 under MM.  f^{UL} = 2.25,
    f^{MD} = 5.5 - 4 = 1.5, f^{LC} = 1.5 + (beta/3) d_{i-1/2}; f^{L,min} = 1 and
    f^{L,max} = min(10, max(2.25, f^{LC}))."""
    S = orc.make_scheme(6, mp_curv=orc.CURV_M4 if curv == "M4" else orc.CURV_MM, mp_beta=beta)
    p = orc.recon_parts(S, np.array([0.0, 0.0, 1.0, 10.0, 27.0, 27.0]))
    assert p["mpmin"] == pytest.approx(1.0, abs=1e-15)
    assert p["mpmax"] == pytest.approx(fmax, rel=1e-15)


def test_tvd5_difference_form_matches_printed_formula(orc):
    S = orc.make_scheme(6, limiter=1)
    rng = np.random.default_rng(31)
    for _ in range(300):
        f = rng.normal(size=6)
        got = orc.recon_parts(S, f)["tvd5"]
        want = tvd5_paper(f[0:5])
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_tvd5_unlimited_is_fifth_order_upwind(orc):
    """Where phi = beta (not clipped), f^{TVD5} = f_i + B/2 is the 5th-order upwind
    linear reconstruction (2, -13, 47, 27, -3)/60 on i-2..i+2."""
    S = orc.make_scheme(6, limiter=1)
    for x0 in np.linspace(0.0, 1.0, 9):
        f, _ = seq_from(lambda x: np.exp(x), 6, i0=x0, h=0.1)
        want = np.dot(np.array([2, -13, 47, 27, -3]) / 60.0, f[0:5])
        assert orc.recon_parts(S, f)["tvd5"] == pytest.approx(want, rel=1e-13)


def test_tvd5_zero_slope_gives_fi(orc):
    S = orc.make_scheme(6, limiter=1)
    f = np.array([0.3, 1.0, 1.0, 2.0, 5.0, 1.0])
    assert orc.recon_parts(S, f)["tvd5"] == 1.0


def test_va_limiter_printed_formula(orc):
    """Eqs. van_Albada_limiter, slop_ratio, vAflux with kappa = 1/3."""
    S = orc.make_scheme(6, limiter=2)
    rng = np.random.default_rng(37)
    for _ in range(100):
        f = rng.normal(size=6)
        fm1, f0, fp1 = f[1], f[2], f[3]
        dm, dp = f0 - fm1, fp1 - f0
        r = dp / dm
        phi = 2 * r / (r * r + 1)
        k = 1.0 / 3.0
        want = f0 + phi / 4 * ((1 - k * phi) * dm + (1 + k * phi) * dp)
        assert orc.recon_parts(S, f)["va"] == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_adaptive_ct_range_and_smooth_limit(orc):
    """TENO8A (Section 2.4): [beta] in {7..10}; for smooth low-wavenumber data eta is ~1,
    m = 0, g = 1 and beta = alpha_1 = 10.5, i.e. C_T = 1e-10.  At a step, m -> 1 and
    beta -> alpha_1 - alpha_2 = 7.  (Parity unpinned beyond these limits.)"""
    S = orc.make_scheme(8)
    f, _ = seq_from(lambda x: x, 8, h=0.1)
    _, _, cte, _, bct = orc.recon(S, f[None, :])
    assert cte[0] == 10 and bct[0] == pytest.approx(10.5)
    ms = np.arange(-3, 5)
    step = np.where(ms <= 0, 1.0, 0.0)
    _, _, cte, _, bct = orc.recon(S, step[None, :])
    assert cte[0] == 7 and bct[0] == pytest.approx(7.0, abs=1e-6)
    rng = np.random.default_rng(41)
    _, _, cte, _, bct = orc.recon(S, rng.normal(size=(200, 8)))
    assert np.all((cte >= 7) & (cte <= 10))
    assert np.all((bct >= 7.0 - 1e-12) & (bct <= 10.5 + 1e-12))


def adaptive_ct_examples():
    """Rows of tests/golden/teno8a_cutoff_examples.txt: (f[8], eta window[4], eta_{i+1/2}, m, g,
    beta, [beta])."""
    out = []
    for r in read_golden("teno8a_cutoff_examples.txt"):
        x = [float(v) for v in r]
        out.append((np.array(x[0:8]), x[8:12], x[12], x[13], x[14], x[15], int(x[16])))
    return out


def test_adaptive_ct_worked_examples(orc):
    """TENO8A's adaptive cutoff between its limits (Section 2.4, Eqs. shock_indicator and
    cut-off_adjust), on sequences worked out by hand from the printed formulas with
    xi = 1e-3, C_r = 0.23, alpha_1 = 10.5, alpha_2 = 3.5 and
    epsilon = 0.9 C_r / (1 - 0.9 C_r) xi^2 = 207/793000000 ~ 2.6103e-7.

    First example, f_{i-3..i+4} = (0, 29, 30, 48, 64, 82, 90, 130) x 1e-4:
      differences Delta f_{i-5/2 .. i+7/2} = (29, 1, 18, 16, 18, 8, 40) x 1e-4;
      eta_{i-1} = (2*1*18e-8 + eps) / ((1 + 324)e-8 + eps) = 49248/278425 = 0.17688067,
      eta_i = eta_{i+1} = (2*18*16e-8 + eps) / ((324 + 256)e-8 + eps) = 0.99340047,
      eta_{i+2} = (2*18*8e-8 + eps) / ((324 + 64)e-8 + eps) = 0.75851442;
      eta_{i+1/2} = min = 0.17688067 (below C_r, so m > 0),
      m = 1 - 0.17688067 / 0.23 = 0.23095362,
      g = (1 - m)^4 (1 + 4m) = 0.34979855 * 1.92381447 = 0.67293532,
      beta = 10.5 - 3.5 (1 - 0.67293532) = 9.35527361, [beta] = 9, C_T = 1e-9.
    The points just outside the window have eta_{i-2} = 0.0969 and eta_{i+3} = 0.394, so
    a window shifted by one gives another eta_{i+1/2} ([beta] 7 or 10); epsilon with xi
    in place of xi^2 makes every eta ~1 ([beta] = 10); (1 - m)^3 in g gives [beta] = 10.
    The second row of the golden file lands on [beta] = 8 the same way.  The oracle must
    reproduce beta to rounding and [beta] exactly."""
    S = orc.make_scheme(8)
    ex = adaptive_ct_examples()
    assert len(ex) == 2
    for f, etas, eh, m, g, beta, ib in ex:
        # the golden rows are consistent with themselves: the chain of printed formulas
        assert eh == pytest.approx(min(etas), rel=1e-13)
        assert m == pytest.approx(1.0 - eh / 0.23, rel=1e-13)
        assert g == pytest.approx((1 - m) ** 4 * (1 + 4 * m), rel=1e-13)
        assert beta == pytest.approx(10.5 - 3.5 * (1 - g), rel=1e-14)
        assert ib == int(np.floor(beta)) and ib in (8, 9)
        _, _, cte, _, bct = orc.recon(S, f[None, :])
        assert cte[0] == ib
        assert bct[0] == pytest.approx(beta, rel=1e-13, abs=0)
        # the f- side reconstructs the sequence mirrored about x_{i+1/2} (f'_m = f_{1-m});
        # its eta'_j is eta_{1-j}, so its window {eta'_{i-1..i+2}} is the same set of values
        _, _, cte_m, _, bct_m = orc.recon(S, f[::-1][None, :].copy())
        assert cte_m[0] == ib and bct_m[0] == pytest.approx(beta, rel=1e-13, abs=0)


@pytest.mark.parametrize("K", [6, 8])
def test_recon_mirror_and_scaling(orc, K):
    """The reconstruction is homogeneous of degree 1 (every stage is scale-covariant) and
    commutes with adding a constant."""
    S = orc.make_scheme(K)
    rng = np.random.default_rng(43)
    v = rng.normal(size=(100, K))
    a, b0, _, _, _ = orc.recon(S, v)
    b, b1, _, _, _ = orc.recon(S, 4.0 * v)
    c, b2, _, _, _ = orc.recon(S, v + 8.0)
    np.testing.assert_array_equal(b0, b1)
    np.testing.assert_allclose(b, 4.0 * a, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(c, a + 8.0, rtol=1e-12, atol=1e-9)
