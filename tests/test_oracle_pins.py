"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it pins and why a plausible mistake would fail it.
None of these re-types the oracle's own formula: they use closed forms,
textbook identities, library special functions, brute force and invariants.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import ndtr, ndtri

import oracle
import workloads


# ----------------------------------------------------------- generators (KAT)

def test_philox_known_answers():
    """Philox-4x32-10 known-answer vectors published with Random123 (Salmon et al. 2011)."""
    assert [int(v) for v in oracle.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert [int(v) for v in oracle.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2)] == \
        [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert [int(v) for v in oracle.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344],
                                                 [0xa4093822, 0x299f31d0])] == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_splitmix64_reference_outputs():
    """First outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014 reference stream)."""
    assert [oracle.splitmix64(0, k) for k in (1, 2, 3)] == \
        [0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f]


def test_normal_cdf_and_inverse_against_library():
    for x in (-37.0, -8.0, -1.3, 0.0, 0.4, 5.0):
        assert oracle.norm_cdf(x) == pytest.approx(float(ndtr(x)), rel=2e-12, abs=1e-300)
    for p in (1e-300, 1e-30, 1e-7, 0.02, 0.5, 0.93, 1 - 1e-10):
        assert oracle.norm_ppf(p) == pytest.approx(float(ndtri(p)), rel=1e-12, abs=1e-14)


# ------------------------------------------------------------------- kernels

def test_kernel_values():
    """RBF sigma^2 exp(-|d|^2/(2 l^2)) (Sec. 3) and Matern-5/2 closed form at known distances."""
    ell = np.array([0.5, 0.5, 0.5])
    a = np.zeros(3); b = np.array([0.5, 0.0, 0.0])
    assert oracle.kernel(oracle.SE, ell, 2.0, a, b) == pytest.approx(2.0 * math.exp(-0.5), rel=1e-15)
    # anisotropy divides each axis by its own length
    assert oracle.kernel(oracle.SE, np.array([1.0, 0.25, 1.0]), 1.0, a, np.array([0.0, 0.25, 0.0])) == \
        pytest.approx(math.exp(-0.5), rel=1e-15)
    r1 = (1 + math.sqrt(5) + 5 / 3) * math.exp(-math.sqrt(5))
    assert oracle.kernel(oracle.MATERN52, ell, 1.0, a, b) == pytest.approx(r1, rel=1e-15)
    assert oracle.kernel(oracle.MATERN52, ell, 3.0, a, a) == 3.0


# ----------------------------------------------------------------- posterior

def test_posterior_single_observation_closed_form():
    """m = 1: mu = k y/(s2+n2), var = s2 - k^2/(s2+n2) (Gaussian conditioning by hand)."""
    X = np.array([[0.3, 0.4, 0.5]]); y = np.array([1.7])
    M = oracle.Model(X, y, oracle.SE, (0.2, 0.3, 0.4), sf2=1.5, sn2=0.1)
    P = np.array([[0.35, 0.2, 0.6], [0.3, 0.4, 0.5]])
    mu, var, cov = M.posterior(P, full_cov=True)
    k = np.array([1.5 * math.exp(-0.5 * ((0.05 / 0.2) ** 2 + (0.2 / 0.3) ** 2 + (0.1 / 0.4) ** 2)), 1.5])
    np.testing.assert_allclose(mu, k * 1.7 / 1.6, rtol=1e-14)
    np.testing.assert_allclose(var, 1.5 - k ** 2 / 1.6, rtol=1e-13)
    k01 = 1.5 * math.exp(-0.5 * ((0.05 / 0.2) ** 2 + (0.2 / 0.3) ** 2 + (0.1 / 0.4) ** 2))
    assert cov[0, 1] == pytest.approx(k01 - k[0] * k[1] / 1.6, rel=1e-13)


def test_posterior_two_observations_closed_form():
    """m = 2: explicit 2x2 inverse of [[s+n, c],[c, s+n]] -- catches a transposed or dropped term."""
    X = np.array([[0.2, 0.5, 0.5], [0.45, 0.5, 0.5]]); y = np.array([0.3, -1.1])
    s2, n2, l = 1.0, 0.05, 0.25
    M = oracle.Model(X, y, oracle.SE, (l, l, l), sf2=s2, sn2=n2)
    x = np.array([[0.3, 0.55, 0.45]])
    mu, var = M.posterior(x)
    kf = lambda a, b: s2 * math.exp(-0.5 * np.sum((a - b) ** 2) / l ** 2)
    c = kf(X[0], X[1]); det = (s2 + n2) ** 2 - c ** 2
    inv = np.array([[s2 + n2, -c], [-c, s2 + n2]]) / det
    k = np.array([kf(x[0], X[0]), kf(x[0], X[1])])
    assert mu[0] == pytest.approx(k @ inv @ y, rel=1e-13)
    assert var[0] == pytest.approx(s2 - k @ inv @ k, rel=1e-12)


def test_posterior_brute_force_small():
    """m <= 20: oracle (Cholesky, forward substitution) vs an LU solve of the joint Gaussian."""
    w = workloads.small(7, 20, 5)
    M = oracle.Model.from_workload(w)
    rng = np.random.default_rng(11)
    P = rng.random((6, 3))
    mu, var, cov = M.posterior(P, full_cov=True)
    # joint covariance of [f(P); y] then Gaussian conditioning with numpy's LU solver
    allx = np.vstack([P, w.X])
    d2 = (((allx[:, None, :] - allx[None, :, :]) / np.array(w.ell)) ** 2).sum(-1)
    Kall = w.sf2 * np.exp(-0.5 * d2)
    Kpp, Kpx, Kxx = Kall[:6, :6], Kall[:6, 6:], Kall[6:, 6:] + w.sn2 * np.eye(20)
    mu_ref = Kpx @ np.linalg.solve(Kxx, w.y)
    cov_ref = Kpp - Kpx @ np.linalg.solve(Kxx, Kpx.T)
    np.testing.assert_allclose(mu, mu_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(cov, cov_ref, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(var, np.diag(cov_ref), rtol=1e-9, atol=1e-12)


def test_interpolation_at_noise_free_observations():
    """sn2 -> 0: mu(x_i) = y_i and var(x_i) ~ 0 (Sec. 3: posterior conditioned on observations)."""
    w = workloads.small(3, 12, 5, ell=(0.15, 0.15, 0.15))
    M = oracle.Model(w.X, w.y, oracle.SE, w.ell, 1.0, 1e-12)
    mu, var = M.posterior(w.X)
    np.testing.assert_allclose(mu, w.y, atol=1e-7)
    assert np.all(np.abs(var) < 1e-8)


def test_variance_nonnegative_and_prior_far_away():
    w = workloads.config1()
    M = oracle.Model.from_workload(w)
    rng = np.random.default_rng(5)
    P = rng.random((400, 3))
    mu, var = M.posterior(P)
    assert np.all(var >= -1e-12) and np.all(var <= w.sf2 + 1e-12)
    # far from every observation the posterior returns to the prior N(0, sf2)
    mu_far, var_far = M.posterior(np.array([[40.0, 40.0, 40.0]]))
    assert abs(mu_far[0]) < 1e-300 + 1e-12 and var_far[0] == pytest.approx(w.sf2, abs=1e-14)


def test_sgpr_equation1_reduces_to_plain_gpr():
    """Eq. (1) with mu_M = K Kt^-1 y and A_M = K - K Kt^-1 K equals plain GPR (the identity used
    to read the paper's SGPR inference for a plain GPR model)."""
    rng = np.random.default_rng(2)
    X = rng.random((10, 3)); y = rng.standard_normal(10)
    M = oracle.Model(X, y, oracle.SE, (0.3, 0.3, 0.3), 1.0, 0.01)
    d2 = (((X[:, None] - X[None]) / 0.3) ** 2).sum(-1)
    K = np.exp(-0.5 * d2); Kt = K + 0.01 * np.eye(10)
    muM = K @ np.linalg.solve(Kt, y); AM = K - K @ np.linalg.solve(Kt, K)
    P = rng.random((5, 3))
    mu1, cov1 = M.posterior_sgpr(muM, AM, P)
    mu2, var2, cov2 = M.posterior(P, full_cov=True)
    np.testing.assert_allclose(mu1, mu2, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(cov1, cov2, rtol=1e-6, atol=1e-9)
    # and the latent posterior at the observations matches mu_M, diag(A_M) (Sec. 5.3 p-test input)
    f = M.factors()
    np.testing.assert_allclose(f["mu_obs"], muM, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(f["var_obs"], np.maximum(np.diag(AM), 1e-12), rtol=1e-6, atol=1e-12)


def _se_np(A, B, ell):
    d = (A[:, None, :] - B[None, :, :]) / np.asarray(ell, float)
    return np.exp(-0.5 * (d ** 2).sum(-1))


def test_sgpr_model_with_exact_inducing_distribution_equals_plain_gpr():
    """An SGPR model (Eq. 1 with a stored N(mu_M, A_M)) whose inducing points are the observations
    and whose distribution is their exact latent posterior (mu_M = K Kt^-1 y, A_M = K - K Kt^-1 K,
    computed here with a dense NumPy solve) reproduces the plain GPR model: the 15 per-point
    statistics, the cell LCP, and the p-test inputs (Sec. 5.3: mu_M and diag A_M)."""
    rng = np.random.default_rng(12)
    X = rng.random((24, 3)); y = rng.standard_normal(24)
    ell, sn2 = (0.3, 0.35, 0.4), 1e-2
    K = _se_np(X, X, ell); Kt = K + sn2 * np.eye(24)
    muM = K @ np.linalg.solve(Kt, y); AM = K - K @ np.linalg.solve(Kt, K); AM = 0.5 * (AM + AM.T)
    plain = oracle.Model(X, y, oracle.SE, ell, 1.0, sn2)
    sg = oracle.Model.sgpr(X, muM, AM, oracle.SE, ell, 1.0, 0.0)
    a = sg.stats15(7); b = plain.stats15(7)
    ok = ~np.isnan(b)
    assert np.array_equal(ok, ~np.isnan(a))
    np.testing.assert_allclose(a[ok], b[ok], rtol=1e-7, atol=1e-9)
    th = float(np.median(y))
    np.testing.assert_allclose(sg.lcp_dense(7, th), plain.lcp_dense(7, th), atol=1e-7)
    f = sg.factors()
    np.testing.assert_array_equal(f["mu_obs"], muM)
    np.testing.assert_array_equal(f["var_obs"], np.maximum(np.diag(AM), 1e-12))


def test_sgpr_terms_special_cases():
    """Each term of Eq. 1 in isolation (jitter 0): with A_M = 0 the inducing values are known, so the
    posterior interpolates them (mu(x_i) = mu_M,i, var(x_i) = 0: the second term cancels the prior);
    with A_M = K_MM and mu_M = 0 they carry no information, so the posterior is the prior
    (mu = 0, Sigma = K_II: the third term cancels the second)."""
    rng = np.random.default_rng(13)
    X = rng.random((12, 3)); ell = (0.35, 0.35, 0.35)
    K = _se_np(X, X, ell)
    muM = rng.standard_normal(12)
    known = oracle.Model.sgpr(X, muM, np.zeros((12, 12)), oracle.SE, ell, 1.0, 0.0)
    mu, var = known.posterior(X)
    np.testing.assert_allclose(mu, muM, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(var, 0.0, atol=1e-8)
    blind = oracle.Model.sgpr(X, np.zeros(12), K, oracle.SE, ell, 1.0, 0.0)
    P = rng.random((6, 3))
    mu, var, cov = blind.posterior(P, full_cov=True)
    np.testing.assert_allclose(mu, 0.0, atol=1e-12)
    np.testing.assert_allclose(cov, _se_np(P, P, ell), atol=1e-8)


def test_sgpr_bound_gradient_matches_finite_differences():
    """The regional bound's g = side (theta - mu) / sigma on an SGPR model: its gradient (through
    Eq. 1: d mu = dk^T K_MM^-1 mu_M, d var = -2 dk^T (K_MM^-1 k - K_MM^-1 A_M K_MM^-1 k)) against central
    differences, and g against the posterior at the point."""
    w = workloads.sgpr(seed=3, m=60, n_train=400, n=9)
    M = oracle.Model.from_workload(w)
    th = w.isovalues[1]
    x = np.array([[0.43, 0.31, 0.57]])
    for side in (1, -1):
        g, gr = M.eval_g(x, th, side)
        for d in range(3):
            e = np.zeros(3); e[d] = 1e-6
            gp, _ = M.eval_g(x + e, th, side); gm, _ = M.eval_g(x - e, th, side)
            assert gr[0, d] == pytest.approx((gp[0] - gm[0]) / 2e-6, rel=1e-5, abs=1e-5)
        mu, var = M.posterior(x)
        assert g[0] == pytest.approx(side * (th - mu[0]) / math.sqrt(var[0]), rel=1e-12)


def test_stats15_match_full_covariance():
    """The 15 per-point stats equal the entries of the joint posterior of the point and its
    13 forward neighbours, and cover every corner pair of a cell."""
    w = workloads.small(4, 30, 9)
    M = oracle.Model.from_workload(w)
    st = M.stats15(9, (2, 3, 1), (5, 6, 4))
    offs = [(1, -1, -1), (1, -1, 0), (1, -1, 1), (1, 0, -1), (1, 0, 0), (1, 0, 1), (1, 1, -1), (1, 1, 0),
            (1, 1, 1), (0, 1, -1), (0, 1, 0), (0, 1, 1), (0, 0, 1)]
    # every nonzero difference of two cell corners is +- one of the 13 offsets
    diffs = {tuple(np.array(a) - np.array(b)) for a in np.ndindex(2, 2, 2) for b in np.ndindex(2, 2, 2) if a != b}
    assert all(d in offs or tuple(-np.array(d)) in offs for d in diffs) and len(offs) == 13
    h = 1.0 / 8
    p = 0
    for c in range(1, 4):
        for b in range(3, 6):
            for a in range(2, 5):
                pts = [(a, b, c)] + [(a + o[0], b + o[1], c + o[2]) for o in offs]
                mu, var, cov = M.posterior(np.array(pts, float) * h, full_cov=True)
                assert st[p, 0] == pytest.approx(mu[0], rel=1e-12, abs=1e-13)
                assert st[p, 1] == pytest.approx(var[0], rel=1e-9, abs=1e-14)
                np.testing.assert_allclose(st[p, 2:], cov[0, 1:], rtol=1e-9, atol=1e-14)
                p += 1


# --------------------------------------------------------- cell LCP (Sec. 4)

def _shift(seed=0, d=8):
    return np.array([oracle.splitmix64(seed, i + 1) >> 32 for i in range(d - 1)], np.uint32)


def test_lcp_independent_corners_closed_form():
    """Diagonal Sigma: P(all<t) = prod Phi(z_c) exactly (SOV is exact when L is diagonal)."""
    rng = np.random.default_rng(1)
    mu = rng.normal(0, 0.5, 8); sd = rng.uniform(0.3, 1.0, 8); th = 0.1
    S = np.diag(sd ** 2)
    lcp = oracle.cell_lcp(mu, S, th, tau=0.0, n_samples=64)
    ref = 1 - np.prod(ndtr((th - mu) / sd)) - np.prod(ndtr((mu - th) / sd))
    assert lcp == pytest.approx(ref, abs=1e-13)
    assert oracle.cell_lcp(mu, S, th, est=oracle.EST_SOV_ORD, tau=0.0, n_samples=64) == pytest.approx(ref, abs=1e-13)


def test_lcp_equicorrelated_quadrature():
    """rho >= 0 equicorrelated, equal mean/variance: P(all<t) = int phi(s) Phi((z+sqrt(rho)s)/sqrt(1-rho))^8 ds."""
    rho, z = 0.6, 0.3
    S = np.full((8, 8), rho) + (1 - rho) * np.eye(8)
    f = lambda s, zz: math.exp(-s * s / 2) / math.sqrt(2 * math.pi) * ndtr((zz + math.sqrt(rho) * s) / math.sqrt(1 - rho)) ** 8
    plo = integrate.quad(f, -12, 12, args=(z,), epsabs=1e-14)[0]
    phi = integrate.quad(f, -12, 12, args=(-z,), epsabs=1e-14)[0]
    ref = 1 - plo - phi
    lcp = oracle.cell_lcp(np.zeros(8), S, z, tau=0.0, n_samples=1 << 16)
    assert lcp == pytest.approx(ref, abs=2e-5)
    lcp1600 = oracle.cell_lcp(np.zeros(8), S, z, tau=0.0, n_samples=1600)
    assert lcp1600 == pytest.approx(ref, abs=2e-3)


def test_lcp_rho_half_exact():
    """rho = 1/2, mu = theta: P(all 8 < theta) = 1/9 exactly, so LCP = 7/9."""
    S = np.full((8, 8), 0.5) + 0.5 * np.eye(8)
    lcp = oracle.cell_lcp(np.zeros(8), S, 0.0, tau=0.0, n_samples=1 << 16)
    assert lcp == pytest.approx(7 / 9, abs=2e-5)


def test_orthant_d2_d3_arcsine():
    """d = 2: 1/4 + asin(rho)/(2 pi);  d = 3: 1/8 + sum asin(rho_ij)/(4 pi)  (Sheppard's formulas)."""
    r = 0.37
    L2 = np.linalg.cholesky(np.array([[1, r], [r, 1.0]]))
    assert oracle.sov_orthant(L2, np.zeros(2), 1 << 15, _shift(3, 2)) == pytest.approx(0.25 + math.asin(r) / (2 * math.pi), abs=1e-6)
    R = np.array([[1, 0.2, -0.3], [0.2, 1, 0.5], [-0.3, 0.5, 1.0]])
    L3 = np.linalg.cholesky(R)
    ref = 0.125 + (math.asin(0.2) + math.asin(-0.3) + math.asin(0.5)) / (4 * math.pi)
    assert oracle.sov_orthant(L3, np.zeros(3), 1 << 15, _shift(3, 3)) == pytest.approx(ref, abs=2e-5)
    # through the cell rule with d = 3: LCP = 1 - 2 P(orthant)
    assert oracle.cell_lcp(np.zeros(3), R, 0.0, tau=0.0, n_samples=1 << 15) == pytest.approx(1 - 2 * ref, abs=4e-5)


def test_lcp_perfect_correlation_vanishes():
    """All corners perfectly correlated (one variable): the field never crosses inside the cell."""
    S = np.full((8, 8), 0.04)
    assert oracle.cell_lcp(np.full(8, 0.1), S, 0.1, tau=1e-10, n_samples=1600) < 1e-3


def test_lcp_mc_agrees_with_sov():
    """Paper's MC estimator (Sec. 4, 1600 samples, Sec. 6.4) agrees with SOV within its standard error."""
    rng = np.random.default_rng(9)
    A = rng.normal(size=(8, 8)); S = A @ A.T / 8 + 0.2 * np.eye(8)
    mu = rng.normal(0, 0.3, 8)
    sov = oracle.cell_lcp(mu, S, 0.0, tau=0.0, n_samples=1 << 15)
    for n, tol in ((1600, 4.0), (200000, 4.0)):
        mc = oracle.cell_lcp(mu, S, 0.0, est=oracle.EST_MC, tau=0.0, n_samples=n, cell=17)
        se = math.sqrt(sov * (1 - sov) / n)
        assert abs(mc - sov) < tol * se + 1e-12


def _corner_se_cov(h_over_l, aniso=(1.0, 1.3, 0.8)):
    """SE covariance of the 8 corners of a unit cell (x-fastest corner order), spacing h / l per axis."""
    c = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], float)
    d = (c[:, None, :] - c[None, :, :]) * h_over_l / np.array(aniso)
    return np.exp(-0.5 * (d ** 2).sum(-1))


def test_sov_general_cells_against_genz_mvn_cdf():
    """Sec. 4's cell LCP, 1 - P(all corners < theta) - P(all > theta), on general 8-variate cells:
    random SPD covariances and SE corner covariances with a small nugget (condition numbers up to
    7e4, like the strongly correlated corners of a fine grid).  The two orthants are 8-D normal
    CDFs, which SciPy evaluates by Genz's own randomised lattice algorithm (an independent code).
    At 2^20 points the sequential-conditioning rule agrees with it to 6e-5; at the 1600 points of
    the paper's sample count its error stays below a fifth of the standard error of the paper's
    1600-sample Monte Carlo estimator, sqrt(p (1 - p) / 1600).  A transposed or mis-indexed factor,
    a wrong conditional shift or a dropped orthant fails the first check."""
    from scipy.stats import multivariate_normal as mvn
    rng = np.random.default_rng(5)
    cases = []
    A = rng.normal(size=(8, 8)); cases.append((rng.normal(0, 0.3, 8), A @ A.T / 8 + 0.2 * np.eye(8), 0.0))
    A = rng.normal(size=(8, 8)); cases.append((rng.normal(0.2, 0.3, 8), A @ A.T / 8 + 0.05 * np.eye(8), 0.1))
    cases.append((rng.normal(0, 0.1, 8), _corner_se_cov(0.5) + 1e-3 * np.eye(8), 0.05))
    cases.append((np.linspace(-0.05, 0.05, 8), _corner_se_cov(0.2) + 1e-4 * np.eye(8), 0.0))
    cases.append((rng.normal(0.3, 0.2, 8), _corner_se_cov(0.3) + 1e-4 * np.eye(8), 0.0))
    for mu, S, th in cases:
        p_lo = mvn.cdf(np.full(8, th), mean=mu, cov=S, abseps=1e-6, releps=0)
        p_hi = mvn.cdf(np.full(8, -th), mean=-mu, cov=S, abseps=1e-6, releps=0)
        ref = 1.0 - p_lo - p_hi
        big = oracle.cell_lcp(mu, S, th, tau=0.0, n_samples=1 << 20)
        assert big == pytest.approx(ref, abs=6e-5), (big, ref)
        paper_n = oracle.cell_lcp(mu, S, th, tau=0.0, n_samples=1600)
        assert abs(paper_n - ref) <= 0.2 * math.sqrt(ref * (1 - ref) / 1600), (paper_n, ref)
        # the ordered variant integrates the same orthants in another variable order
        big = oracle.cell_lcp(mu, S, th, est=oracle.EST_SOV_ORD, tau=0.0, n_samples=1 << 20)
        assert big == pytest.approx(ref, abs=6e-5), (big, ref)


def test_ordered_sov_perfectly_correlated_corners_closed_form():
    """Corners that share one normal variable, Y_c = mu_c + sigma Z with distinct means:
    P(all < theta) = Phi(min_c z_c), P(all > theta) = Phi(-max_c z_c), z_c = (theta - mu_c) / sigma,
    so LCP = Phi(z_max) - Phi(z_min) (Sec. 4's definition).  The ordered estimator takes the corner
    with the smallest standardised threshold first for the all-below orthant (the largest for the
    all-above one): its first factor is the exact answer and every later factor is 1 up to the
    jitter, whatever the lattice.  A reversed or unsorted order misses by up to ~1e-3 (the index
    order's error here), so the order itself is pinned."""
    rng = np.random.default_rng(3)
    sd = 0.2
    S = np.full((8, 8), sd * sd)
    for trial in range(4):
        mu = rng.normal(0.0, 0.1, 8)
        th = float(np.median(mu)) + 0.01 * trial
        z = (th - mu) / sd
        exact = ndtr(z.max()) - ndtr(z.min())
        got = oracle.cell_lcp(mu, S, th, est=oracle.EST_SOV_ORD, tau=1e-10, n_samples=1600)
        assert got == pytest.approx(exact, abs=1e-8), (got, exact)


def test_ordered_sov_relabelling_invariance():
    """The ordered estimator sorts the corners by their standardised thresholds, so relabelling the
    corners (permuting mu and Sigma together) leaves its factors, and its value, unchanged to the
    last bit; the index-order estimator has no such property."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(8, 8)); S = A @ A.T / 8 + 0.1 * np.eye(8)
    mu = rng.normal(0.0, 0.4, 8); th = 0.05
    a = oracle.cell_lcp(mu, S, th, est=oracle.EST_SOV_ORD, n_samples=1600, cell=5)
    for seed in range(3):
        p = np.random.default_rng(100 + seed).permutation(8)
        b = oracle.cell_lcp(mu[p], S[np.ix_(p, p)], th, est=oracle.EST_SOV_ORD, n_samples=1600, cell=5)
        assert a == b, (a, b)


def test_bivariate_normal_against_library_and_closed_form():
    """P(X1 < a, X2 < b) (the edge estimator's building block): SciPy's multivariate normal CDF over
    random thresholds and correlations up to |r| = 1 - 1e-8, and the orthant 1/4 + asin(r) / (2 pi)."""
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(21)
    for _ in range(120):
        a, b = rng.uniform(-6, 6, 2)
        r = rng.choice([rng.uniform(-0.99, 0.99), 1 - 10 ** rng.uniform(-8, -1), -(1 - 10 ** rng.uniform(-8, -1))])
        ref = multivariate_normal.cdf([a, b], mean=[0, 0], cov=[[1, r], [r, 1]], abseps=1e-13, releps=1e-13)
        assert oracle.bvn_lower(a, b, r) == pytest.approx(ref, abs=1e-12)
    for r in (-0.9, -0.3, 0.0, 0.5, 0.999):
        assert oracle.bvn_lower(0.0, 0.0, r) == pytest.approx(0.25 + math.asin(r) / (2 * math.pi), abs=1e-13)


def test_independent_corner_estimator():
    """The independent-corner closed form equals the exact LCP when the corners are independent
    (diagonal Sigma: the sequential-conditioning estimator is exact there) and ignores the
    off-diagonal entries otherwise."""
    rng = np.random.default_rng(22)
    mu = rng.normal(0, 0.3, 8); d = rng.uniform(0.05, 0.3, 8)
    S = np.diag(d)
    assert oracle.cell_lcp(mu, S, 0.1, est=oracle.EST_INDEP) == pytest.approx(oracle.cell_lcp(mu, S, 0.1), abs=1e-12)
    A = rng.normal(size=(8, 8)); C = A @ A.T / 8
    Sc = C + np.diag(np.diag(S) + 0.02 - np.diag(C))  # same diagonal, correlated
    assert oracle.cell_lcp(mu, Sc, 0.1, est=oracle.EST_INDEP) == \
        pytest.approx(oracle.cell_lcp(mu, np.diag(np.diag(Sc)), 0.1, est=oracle.EST_INDEP), abs=1e-15)


def test_edge_max_estimator():
    """Pothkow et al.'s edge approximation: for two variables it is the exact segment crossing
    probability of Sec. 4's first formula (SciPy's bivariate CDF); for a cell it is the largest of the
    12 edge probabilities and never exceeds the cell's LCP (a crossed edge crosses the cell)."""
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(23)
    mu2 = np.array([0.05, -0.1]); S2 = np.array([[0.04, 0.03], [0.03, 0.05]])
    Sj = S2 + np.eye(2) * 1e-10 * 0.05  # the jittered Sigma (default tau)
    lo = multivariate_normal.cdf([0.0, 0.0], mean=mu2, cov=Sj)
    hi = multivariate_normal.cdf([0.0, 0.0], mean=-mu2, cov=Sj)
    assert oracle.cell_lcp(mu2, S2, 0.0, est=oracle.EST_EDGE) == pytest.approx(1 - lo - hi, abs=1e-9)
    for _ in range(6):
        A = rng.normal(size=(8, 8)); S = A @ A.T / 8 + 0.3 * np.ones((8, 8)) + 0.02 * np.eye(8)
        mu = rng.normal(0, 0.3, 8)
        e = oracle.cell_lcp(mu, S, 0.05, est=oracle.EST_EDGE)
        full = oracle.cell_lcp(mu, S, 0.05, n_samples=20000)
        assert e <= full + 1e-3
        Sj = S + np.eye(8) * 1e-10 * np.max(np.diag(S))
        best = 0.0
        for i in range(8):
            for a in range(3):
                j = i ^ (1 << a)
                if j < i:
                    continue
                C = Sj[np.ix_([i, j], [i, j])]
                p_lo = multivariate_normal.cdf([0.05, 0.05], mean=mu[[i, j]], cov=C, abseps=1e-12)
                p_hi = multivariate_normal.cdf([-0.05, -0.05], mean=-mu[[i, j]], cov=C, abseps=1e-12)
                best = max(best, 1 - p_lo - p_hi)
        assert e == pytest.approx(best, abs=1e-9)


def test_lcp_skip_and_range():
    """LCP in [0,1]; the Boole pre-skip returns exactly 0 far from theta; deterministic cells."""
    S = 0.01 * (np.full((8, 8), 0.9) + 0.1 * np.eye(8))
    assert oracle.cell_lcp(np.full(8, 5.0), S, 0.0) == 0.0
    assert oracle.cell_lcp(np.linspace(-1, 1, 8), np.zeros((8, 8)), 0.05) == 1.0
    assert oracle.cell_lcp(np.full(8, 2.0), np.zeros((8, 8)), 0.05) == 0.0
    rng = np.random.default_rng(4)
    for _ in range(20):
        A = rng.normal(size=(8, 8)); S = A @ A.T * rng.uniform(0.001, 1)
        v = oracle.cell_lcp(rng.normal(0, 1, 8), S, 0.0)
        assert 0.0 <= v <= 1.0
    # a corner variance that is negative even after the jitter: no Gaussian, so no LCP
    Sn = S.copy(); Sn[3, 3] = -0.5 * Sn.diagonal().max()
    for est in (oracle.EST_SOV, oracle.EST_MC, oracle.EST_INDEP, oracle.EST_EDGE):
        assert np.isnan(oracle.cell_lcp(np.zeros(8), Sn, 0.0, est=est))


def test_lcp_field_brute_force_mc_small():
    """Dense LCP of a few real cells (Sec. 4): SOV agrees with a brute-force numpy MC of the same
    8-variate posterior, built from full joint covariance by an independent route."""
    w = workloads.config1()
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    n = w.n
    lcp = M.lcp_block(n, th, (10, 10, 10), (14, 12, 11), tau=1e-4)
    rng = np.random.default_rng(0)
    h = 1 / (n - 1)
    idx = 0
    for c in range(10, 11):
        for b in range(10, 12):
            for a in range(10, 14):
                pts = np.array([(a + (q & 1), b + ((q >> 1) & 1), c + (q >> 2)) for q in range(8)], float) * h
                mu, var, cov = M.posterior(pts, full_cov=True)
                cov = cov + 1e-4 * np.max(np.diag(cov)) * np.eye(8)
                Y = rng.multivariate_normal(mu, cov, size=200000, method="eigh")
                mc = 1 - np.mean(np.all(Y < th, 1)) - np.mean(np.all(Y > th, 1))
                assert abs(lcp[idx] - mc) < 4 * math.sqrt(max(mc * (1 - mc), 1e-6) / 200000) + 2e-3
                idx += 1


# ------------------------------------------------- bound + octree (Sec. 5)

def test_eval_g_gradient_matches_finite_differences():
    w = workloads.small(5, 40, 9)
    M = oracle.Model.from_workload(w)
    x = np.array([[0.41, 0.37, 0.52]])
    th = w.isovalues[0]
    for side in (1, -1):
        g, gr = M.eval_g(x, th, side)
        for d in range(3):
            e = np.zeros(3); e[d] = 1e-6
            gp, _ = M.eval_g(x + e, th, side); gm, _ = M.eval_g(x - e, th, side)
            assert gr[0, d] == pytest.approx((gp[0] - gm[0]) / 2e-6, rel=1e-5, abs=1e-6)
        mu, var = M.posterior(x)
        assert g[0] == pytest.approx(side * (th - mu[0]) / math.sqrt(var[0]), rel=1e-12)


def test_bound_dominates_true_regional_lcp():
    """Eq. (upper_bound) is an upper bound: on small nodes (3^3 grid points) where the minimiser is
    exact, the true regional crossing probability (MC over all d points) never exceeds it.  Boole
    gives this with no correlation assumption when the bound is small (1-(1-q)^d <= d q)."""
    w = workloads.small(6, 40, 17, ell=(0.25, 0.25, 0.25))
    M = oracle.Model.from_workload(w)
    D = 4
    l = D - 1  # nodes of 2x2x2 cells = 3^3 grid points
    nodes = np.array([i | (j << 21) | (k << 42) for k in range(8) for j in range(8) for i in range(8)], np.int64)
    th = w.isovalues[0]
    dec, bnd, side = M.octree_level(17, D, l, th, nodes, alpha=1e-3)
    rng = np.random.default_rng(1)
    checked = 0
    for q in np.nonzero(dec == 2)[0][:6].tolist() + np.nonzero(dec == 0)[0][:6].tolist():
        i, j, k = nodes[q] & 0x1FFFFF, (nodes[q] >> 21) & 0x1FFFFF, (nodes[q] >> 42) & 0x1FFFFF
        pts = np.array([(2 * i + a, 2 * j + b, 2 * k + c) for c in range(3) for b in range(3) for a in range(3)], float) / 16
        mu, var, cov = M.posterior(pts, full_cov=True)
        Y = rng.multivariate_normal(mu, cov + 1e-12 * np.eye(27), size=100000, method="eigh")
        sides = side[q]
        if sides == 1:
            p_true = 1 - np.mean(np.all(Y < th, 1))
        elif sides == 2:
            p_true = 1 - np.mean(np.all(Y > th, 1))
        else:
            p_true = 1 - np.mean(np.all(Y < th, 1)) - np.mean(np.all(Y > th, 1))
        assert p_true <= bnd[q] + 4 * math.sqrt(max(bnd[q], 1e-5) / 100000) + 1e-9
        checked += 1
    assert checked >= 6


def _brute_box(M, th, side, lo, hi, n=41):
    t = np.linspace(0, 1, n)
    pts = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3) * (hi - lo) + lo
    g, _ = M.eval_g(pts, th, side)
    return g.min(), pts[np.argmin(g)]


def _polish(M, th, side, lo, hi, x0):
    """L-BFGS-B (the paper's minimiser, Sec. 5.1) from x0 inside the box, via SciPy."""
    from scipy.optimize import minimize
    r = minimize(lambda z: M.eval_g(z, th, side)[0][0], x0, jac=lambda z: M.eval_g(z, th, side)[1][0],
                 method="L-BFGS-B", bounds=list(zip(lo, hi)))
    return float(r.fun)


def test_minimiser_vs_brute_force_lattice():
    """The continuous-box minimiser of the regional bound (Sec. 5.1; the paper minimises with
    L-BFGS-B, the oracle with a 3x3x3 lattice start and T projected steps) on nodes of 5^3 and 9^3
    grid points, both sides:
      - the point it reports lies in the node box and g there equals the value it reports;
      - the value is never above the lattice start and never below the box minimum (a 41^3
        brute-force lattice, and L-BFGS-B polished from the reported point, both bound it);
      - on nodes whose minimum is interior, the projected steps close at least half of the gap
        between the lattice start and the box minimum.
    A flipped step sign (u = +grad g * w) never accepts a step and fails the last check; an
    unclamped step leaves the box; a step evaluated at one point but kept at another breaks the
    value-at-point check."""
    w = workloads.small(8, 40, 17, ell=(0.3, 0.3, 0.3))
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    n, D = 17, 4
    improved, checked = 0, 0
    for l, nodes in ((2, [(0, 0, 0), (2, 0, 0), (0, 1, 0), (1, 1, 0), (3, 2, 1), (2, 2, 1), (1, 0, 1)]),
                     (1, [(0, 0, 0), (1, 1, 1), (0, 1, 0)])):
        for (i, j, k) in nodes:
            node = i | (j << 21) | (k << 42)
            for side in (1, -1):
                v, x, lo, hi = M.node_min(n, D, l, node, th, side)
                assert np.all(hi - lo > 0) and (hi[0] - lo[0]) * 16 == pytest.approx(1 << (D - l))
                assert np.all(x >= lo) and np.all(x <= hi)
                gx, _ = M.eval_g(x, th, side)
                assert gx[0] == pytest.approx(v, rel=1e-12, abs=1e-12)
                lat = np.array([lo + (hi - lo) * np.array(c) / 2 for c in np.ndindex(3, 3, 3)])
                g_lat = M.eval_g(lat, th, side)[0].min()
                g_brute, x_brute = _brute_box(M, th, side, lo, hi)
                g_true = min(g_brute, _polish(M, th, side, lo, hi, x), _polish(M, th, side, lo, hi, x_brute))
                assert v <= g_lat + 1e-12
                assert v >= g_true - 1e-9
                checked += 1
                if g_lat - g_true > 1e-3 and v < g_lat - 1e-9:
                    improved += 1
    assert checked == 20
    assert improved >= 10
    # interior minima: the steps must do real work here (values measured with the 41^3 lattice)
    for l, (i, j, k), side in ((2, (2, 0, 0), -1), (2, (0, 1, 0), -1), (2, (3, 2, 1), 1), (2, (2, 2, 2), 1),
                             (1, (0, 0, 0), -1), (1, (1, 1, 1), 1)):
        node = i | (j << 21) | (k << 42)
        v, x, lo, hi = M.node_min(n, D, l, node, th, side)
        g_lat = M.eval_g(np.array([lo + (hi - lo) * np.array(c) / 2 for c in np.ndindex(3, 3, 3)]), th, side)[0].min()
        g_brute, x_brute = _brute_box(M, th, side, lo, hi)
        assert np.all((x_brute > lo) & (x_brute < hi))  # the brute-force minimum is interior
        assert (g_lat - v) >= 0.5 * (g_lat - g_brute)


def test_minimiser_small_nodes_take_the_exact_grid_minimum():
    """Nodes with at most 3 grid points per axis: the minimum over their grid points (brute force
    over the 27 points, Sec. 5.1's min over D), and the reported point is one of them."""
    w = workloads.small(8, 40, 17, ell=(0.3, 0.3, 0.3))
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    for (i, j, k) in ((0, 0, 0), (3, 5, 2), (7, 7, 7), (4, 1, 6)):
        node = i | (j << 21) | (k << 42)
        for side in (1, -1):
            v, x, lo, hi = M.node_min(17, 4, 3, node, th, side)
            pts = np.array([lo + (hi - lo) * np.array(c) / 2 for c in np.ndindex(3, 3, 3)])
            g = M.eval_g(pts, th, side)[0]
            assert v == g.min()
            assert np.min(np.abs(pts - x).sum(1)) == 0.0


def _np_gp(X, y, ell, sn2):
    """Plain GPR from its definition with a dense inverse (NumPy), independent of the oracle."""
    ell = np.asarray(ell, float)

    def k(A, B):
        d = (A[:, None, :] - B[None, :, :]) / ell
        return np.exp(-0.5 * (d ** 2).sum(-1))
    Q = np.linalg.inv(k(X, X) + sn2 * np.eye(len(y)))

    def post(P):
        ks = k(P, X)
        return ks @ Q @ y, 1.0 - np.einsum("ij,jk,ik->i", ks, Q, ks)
    K = k(X, X)
    mu_M = K @ Q @ y                      # Eq. 1 with the observations as inducing points
    var_M = np.diag(K - K @ Q @ K)
    return post, mu_M, var_M


def _expected_level(X, y, ell, sn2, th, alpha, n, D, l, nodes):
    """Algorithm 1 (Sec. 5.3) for one level, written from the algorithm: p1/p2 from the latent
    posterior at the observations in the closed node box; both > alpha -> subdivide directly;
    p2 <= alpha -> only B_l = min P(Y < theta); p1 <= alpha -> only B_u = min P(Y > theta); no
    observation -> both; bound 1 - B_l^d - B_u^d (Eq. upper_bound, Sec. 5.1) over the node's d grid
    points (nodes of <= 3 points per axis: the exact minimum over them)."""
    from scipy.special import log_ndtr, ndtr
    post, mu_M, var_M = _np_gp(X, y, ell, sn2)
    p_lo = ndtr((th - mu_M) / np.sqrt(var_M))
    p_hi = ndtr((mu_M - th) / np.sqrt(var_M))
    s = 1 << (D - l)
    gx = np.arange(n) / (n - 1)
    out = []
    for nd in nodes:
        ijk = [(nd >> (21 * a)) & 0x1FFFFF for a in range(3)]
        p0 = [c * s for c in ijk]
        p1 = [min((c + 1) * s, n - 1) for c in ijk]
        lo = np.array([gx[a] for a in p0]); hi = np.array([gx[a] for a in p1])
        inside = np.all((X >= lo) & (X <= hi), 1)
        P = np.array([[gx[a], gx[b], gx[c]] for c in range(p0[2], p1[2] + 1)
                      for b in range(p0[1], p1[1] + 1) for a in range(p0[0], p1[0] + 1)])
        mu, var = post(P)
        sd = np.sqrt(var)
        d = len(P)
        has_lo = bool(np.any(p_lo[inside] > alpha)); has_hi = bool(np.any(p_hi[inside] > alpha))
        if inside.any() and has_lo and has_hi:
            out.append((1, None, 0)); continue
        use_lo = (not inside.any()) or not has_hi
        use_hi = (not inside.any()) or not has_lo
        Bl = np.exp(d * log_ndtr(((th - mu) / sd).min())) if use_lo else 0.0
        Bu = np.exp(d * log_ndtr(((mu - th) / sd).min())) if use_hi else 0.0
        bound = 1.0 - Bl - Bu
        side = 0 if (use_lo and use_hi) else (1 if use_lo else 2)
        out.append((2 if bound > alpha else 0, bound, side))
    return out


def test_ptest_side_selection_and_one_sided_bounds():
    """Algorithm 1's p-test with hand-placed observations (theta = 0, alpha = 1e-3, nodes of 3^3
    grid points): node 0 holds an observation far above and one far below theta (direct
    subdivide); node 1 only observations below (p2 <= alpha: lower side only); node 2 only above
    (upper side only); node 3 a dense block of observations below theta (lower side, bound far
    below alpha: dropped); node 6 and 7 share an observation on their common face (closed boxes);
    nodes 4, 5 are empty (both sides).  A swapped lower/upper flag gives node 3 the upper side and
    a bound of 1, and fails."""
    obs = [((0.2, 0.25, 0.25), 2.0), ((0.3, 0.25, 0.3), -2.0), ((0.75, 0.25, 0.25), -3.0),
           ((0.8, 0.3, 0.2), -2.5), ((0.25, 0.75, 0.25), 3.0), ((0.2, 0.8, 0.3), 2.5), ((0.5, 0.75, 0.75), 3.0)]
    obs += [((a, b, c), -3.0) for a in (0.55, 0.75, 0.95) for b in (0.55, 0.75, 0.95) for c in (0.05, 0.25, 0.45)]
    X = np.array([o[0] for o in obs]); y = np.array([o[1] for o in obs])
    ell, sn2, th, alpha = (0.2, 0.2, 0.2), 1e-4, 0.0, 1e-3
    M = oracle.Model(X, y, oracle.SE, ell, 1.0, sn2)
    nodes = np.array([i | (j << 21) | (k << 42) for k in range(2) for j in range(2) for i in range(2)], np.int64)
    dec, bnd, side = M.octree_level(5, 2, 1, th, nodes, alpha=alpha)
    exp = _expected_level(X, y, ell, sn2, th, alpha, 5, 2, 1, nodes)
    for q, (e_dec, e_bnd, e_side) in enumerate(exp):
        assert dec[q] == e_dec, q
        assert side[q] == e_side, q
        if e_bnd is None:
            assert np.isnan(bnd[q])
        else:
            assert bnd[q] == pytest.approx(e_bnd, rel=1e-9, abs=1e-12), q
    assert [int(v) for v in dec[:4]] == [1, 2, 2, 0]
    assert [int(v) for v in side] == [0, 1, 2, 1, 0, 0, 2, 2]
    assert bnd[3] < 1e-10


def test_two_sided_bound_when_the_node_is_empty():
    """An empty node takes both sides, 1 - B_l^d - B_u^d (Eq. upper_bound): with the mean near theta
    over single-cell nodes (d = 8) both terms are ~0.5^8, so dropping either term or using the
    one-sided form moves the bound by ~4e-3."""
    X = np.array([[0.1, 0.1, 0.1], [0.15, 0.12, 0.08]]); y = np.array([0.01, -0.02])
    ell, sn2, th, alpha = (0.5, 0.5, 0.5), 1e-4, 0.0, 1e-3
    M = oracle.Model(X, y, oracle.SE, ell, 1.0, sn2)
    nodes = np.array([i | (j << 21) | (k << 42) for k in range(2) for j in range(2) for i in range(2)], np.int64)
    dec, bnd, side = M.octree_level(3, 1, 1, th, nodes, alpha=alpha)
    exp = _expected_level(X, y, ell, sn2, th, alpha, 3, 1, 1, nodes)
    for q in range(1, 8):
        e_dec, e_bnd, e_side = exp[q]
        assert side[q] == 0 and e_side == 0
        assert bnd[q] == pytest.approx(e_bnd, rel=1e-12, abs=1e-13)
        assert 1e-3 < 1.0 - bnd[q] < 0.1  # both terms matter


def test_local_model_bound_sec52():
    """The local approximation of Sec. 5.2: (i) when beta * l covers the domain the local set is all
    of M and every decision and bound equals the full model's; (ii) for a node whose enlarged box
    (beta * l_d per axis, closed) holds only some observations, the bound is Eq. upper_bound of the
    model built from exactly those observations (selected here with NumPy); (iii) with beta = 0 a
    node holding no observation is bounded by the prior (mu = 0, sigma^2 = sf2)."""
    from scipy.special import log_ndtr
    w = workloads.small(31, 50, 17, ell=(0.08, 0.1, 0.12))
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    n, D = 17, 4
    for l in (1, 2, 3):
        s = 1 << l
        nodes = np.array([i | (j << 21) | (k << 42) for k in range(s) for j in range(s) for i in range(s)], np.int64)
        full = M.octree_level(n, D, l, th, nodes)
        wide = M.octree_level(n, D, l, th, nodes, beta=20.0)
        for a, b in zip(full, wide):
            np.testing.assert_array_equal(a, b)
    # (ii) nodes of 5^3 grid points with a strict local subset
    l, beta, checked = 2, 1.5, 0
    for (i, j, k) in ((0, 0, 0), (3, 1, 2), (1, 3, 3), (2, 2, 0)):
        node = np.array([i | (j << 21) | (k << 42)], np.int64)
        dec, bnd, side = M.octree_level(n, D, l, th, node, beta=beta)
        if dec[0] == 1:
            continue
        lo = np.array([i, j, k]) * 4 / 16; hi = lo + 4 / 16
        ell = np.array(w.ell)
        sel = np.all((w.X >= lo - beta * ell) & (w.X <= hi + beta * ell), 1)
        assert 0 < sel.sum() < w.m
        sub = oracle.Model(w.X[sel], w.y[sel], w.kernel, w.ell, w.sf2, w.sn2)
        lb = {}
        for sd in (1, -1):
            v, _, _, _ = sub.node_min(n, D, l, int(node[0]), th, sd)
            lb[sd] = 125 * log_ndtr(v)
        e = {1: -np.expm1(lb[1]), 2: -np.expm1(lb[-1]), 0: -np.expm1(lb[1]) - np.exp(lb[-1])}[int(side[0])]
        assert bnd[0] == pytest.approx(e, rel=1e-12, abs=1e-14)
        checked += 1
    assert checked >= 2
    # (iii) beta = 0: an empty node's local model is the prior
    for q in range(64):
        i, j, k = q % 4, (q // 4) % 4, q // 16
        lo = np.array([i, j, k]) / 4; hi = lo + 0.25
        if np.any(np.all((w.X >= lo) & (w.X <= hi), 1)):
            continue
        node = np.array([i | (j << 21) | (k << 42)], np.int64)
        dec, bnd, side = M.octree_level(n, D, 2, th, node, beta=0.0)
        z = th / math.sqrt(w.sf2)
        e = -np.expm1(125 * log_ndtr(z)) - np.exp(125 * log_ndtr(-z))
        assert side[0] == 0 and bnd[0] == pytest.approx(e, rel=1e-12, abs=1e-14)
        break
    else:
        pytest.fail("no empty node")


def test_kd_tree_levels():
    """The K-D tree of Sec. 9 halves x, y, z in turn: its level 3L nodes are exactly the octree's
    level-L nodes, so for the same node codes both give the same decisions and bounds; in between, a
    node at level 3L + a spans half of its parent along axis a - 1 (checked through the p-test of a
    node whose half holds no observation).  With alpha -> 0 it keeps every cell of non-zero LCP and
    the adaptive field equals the dense one on S."""
    w = workloads.config2()
    M = oracle.Model.from_workload(w)
    th = w.isovalues[1]
    n, D = 17, 4
    for L in (1, 2, 3):
        s = 1 << L
        nodes = np.array([i | (j << 21) | (k << 42) for k in range(s) for j in range(s) for i in range(s)], np.int64)
        a = M.octree_level(n, D, L, th, nodes)
        b = M.octree_level(n, D, 3 * L, th, nodes, kd=True)
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)
    # level 1: two x-halves; level 2: (x, y) quarters at full z; level 5: (1/4, 1/4, 1/2)
    for l, node, lo, hi in ((1, 1, (0.5, 0, 0), (1, 1, 1)), (2, 1 | (1 << 21), (0.5, 0.5, 0), (1, 1, 1)),
                            (5, 3 | (2 << 21) | (1 << 42), (0.75, 0.5, 0.5), (1, 0.75, 1))):
        _, _, blo, bhi = M.node_min(n, D, l, node, th, 1, kd=True)
        np.testing.assert_allclose(blo, lo, atol=1e-15); np.testing.assert_allclose(bhi, hi, atol=1e-15)
    w2 = workloads.small(2, 30, 9, ell=(0.3, 0.3, 0.3))
    M2 = oracle.Model.from_workload(w2)
    th2 = w2.isovalues[0]
    Dd = workloads.depth_for(9)
    dense = M2.lcp_dense(9, th2)
    field, leaves, levels = M2.lcp_adaptive(9, Dd, th2, alpha=1e-300, kd=True)
    assert len(levels) == 3 * Dd + 1
    assert np.all(field[dense > 1e-12] == dense[dense > 1e-12])
    field3, leaves3, _ = M2.lcp_adaptive(9, Dd, th2, kd=True)
    lin = (leaves3 & 0x1FFFFF) + 8 * (((leaves3 >> 21) & 0x1FFFFF) + 8 * ((leaves3 >> 42) & 0x1FFFFF))
    np.testing.assert_array_equal(field3[lin], dense[lin])


def test_octree_alpha_zero_keeps_nonzero_cells_and_adaptive_equals_dense():
    """Algorithm 1 with alpha -> 0 keeps every cell whose dense LCP is non-zero, and the adaptive
    field equals the dense field on S and is 0 elsewhere (Sec. 5.3, last paragraph)."""
    w = workloads.small(2, 30, 9, ell=(0.3, 0.3, 0.3))
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    D = workloads.depth_for(9)
    dense = M.lcp_dense(9, th)
    field, leaves, levels = M.lcp_adaptive(9, D, th, alpha=1e-300)
    assert np.all(field[dense > 1e-12] == dense[dense > 1e-12])
    field3, leaves3, _ = M.lcp_adaptive(9, D, th, alpha=1e-3)
    lin = (leaves3 & 0x1FFFFF) + 8 * (((leaves3 >> 21) & 0x1FFFFF) + 8 * ((leaves3 >> 42) & 0x1FFFFF))
    np.testing.assert_array_equal(field3[lin], dense[lin])
    mask = np.ones(dense.size, bool); mask[lin] = False
    assert np.all(field3[mask] == 0)
    # RMSE against dense is small, as the paper reports (Sec. 7.2): a sanity range, not a pin
    assert math.sqrt(np.mean((field3 - dense) ** 2)) < 5e-3


# ------------------------------------------------------------ adjoint (no paper counterpart)

def test_cell_adjoint_matches_finite_differences():
    """Reverse sweep through the sequential-conditioning rule and the 8x8 Cholesky: dLCP/dmu and
    dLCP/dSigma against central differences of the same estimator (fixed lattice: smooth)."""
    rng = np.random.default_rng(3)
    A = rng.normal(size=(8, 8)); S = A @ A.T / 8 + 0.05 * np.ones((8, 8)) + 0.02 * np.eye(8)
    mu = rng.normal(0, 0.2, 8)
    v, mb, Sb = oracle.cell_lcp_adj(mu, S, 0.05)
    assert v == pytest.approx(oracle.cell_lcp(mu, S, 0.05), abs=1e-15)
    h = 1e-5
    for i in range(8):
        e = np.zeros(8); e[i] = h
        fd = (oracle.cell_lcp(mu + e, S, 0.05) - oracle.cell_lcp(mu - e, S, 0.05)) / (2 * h)
        assert mb[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for (i, j) in ((0, 0), (2, 5), (7, 7), (1, 6), (3, 4)):
        E = np.zeros((8, 8)); E[i, j] += h
        if i != j:
            E[j, i] += h
        fd = (oracle.cell_lcp(mu, S + E, 0.05) - oracle.cell_lcp(mu, S - E, 0.05)) / (2 * h)
        an = Sb[i, j] + (Sb[j, i] if i != j else 0.0)
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_ordered_cell_adjoint_matches_finite_differences():
    """The ordered rule's reverse sweep (each orthant on its own permuted factor, adjoints permuted
    back): dLCP/dmu and dLCP/dSigma against central differences of the same estimator at a point
    whose corner order does not change within the step (the order is piecewise constant)."""
    rng = np.random.default_rng(3)
    A = rng.normal(size=(8, 8)); S = A @ A.T / 8 + 0.05 * np.ones((8, 8)) + 0.02 * np.eye(8)
    mu = rng.normal(0, 0.2, 8)
    th = 0.05
    z = (th - mu) / np.sqrt(np.diag(S))
    assert np.min(np.diff(np.sort(z))) > 1e-3  # no near-ties: a 1e-5 step keeps both orders
    est = oracle.EST_SOV_ORD
    v, mb, Sb = oracle.cell_lcp_adj(mu, S, th, est=est)
    assert v == pytest.approx(oracle.cell_lcp(mu, S, th, est=est), abs=1e-15)
    h = 1e-5
    for i in range(8):
        e = np.zeros(8); e[i] = h
        fd = (oracle.cell_lcp(mu + e, S, th, est=est) - oracle.cell_lcp(mu - e, S, th, est=est)) / (2 * h)
        assert mb[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for (i, j) in ((0, 0), (2, 5), (7, 7), (1, 6), (3, 4)):
        E = np.zeros((8, 8)); E[i, j] += h
        if i != j:
            E[j, i] += h
        fd = (oracle.cell_lcp(mu, S + E, th, est=est) - oracle.cell_lcp(mu, S - E, th, est=est)) / (2 * h)
        an = Sb[i, j] + (Sb[j, i] if i != j else 0.0)
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # the two rules estimate the same LCP, so their gradients agree to the estimators' accuracy
    _, mb0, _ = oracle.cell_lcp_adj(mu, S, th)
    assert np.abs(mb - mb0).max() <= 0.05 * np.abs(mb0).max()


@pytest.mark.parametrize("kernel", [workloads.SE, workloads.MATERN52])
def test_field_gradient_matches_finite_differences(kernel):
    """loss = sum_c w_c LCP_c on a small field: dloss/dy_i and dloss/dlog l_d (analytic, chain rule
    through Eq. 1, the kernel derivative through r for Matern-5/2) against central differences
    with h = 1e-3."""
    w = workloads.small(5, 30, 9, ell=(0.2, 0.25, 0.3), kernel=kernel)
    M = oracle.Model.from_workload(w)
    th = w.isovalues[0]
    wts = np.random.default_rng(5).random(512)
    loss, dy, dl = M.lcp_grad(9, th, wts)
    assert loss == pytest.approx(float(np.dot(wts, M.lcp_dense(9, th))), rel=1e-12)
    h = 1e-3
    for i in (0, 7, 21):
        y2 = w.y.copy(); y2[i] += h
        lp = oracle.Model(w.X, y2, w.kernel, w.ell, w.sf2, w.sn2).lcp_grad(9, th, wts)[0]
        y2[i] -= 2 * h
        lm = oracle.Model(w.X, y2, w.kernel, w.ell, w.sf2, w.sn2).lcp_grad(9, th, wts)[0]
        assert dy[i] == pytest.approx((lp - lm) / (2 * h), rel=2e-4, abs=1e-6)
    for d in range(3):
        e = np.zeros(3); e[d] = h
        lp = oracle.Model(w.X, w.y, w.kernel, tuple(np.array(w.ell) * np.exp(e)), w.sf2, w.sn2).lcp_grad(9, th, wts)[0]
        lm = oracle.Model(w.X, w.y, w.kernel, tuple(np.array(w.ell) * np.exp(-e)), w.sf2, w.sn2).lcp_grad(9, th, wts)[0]
        assert dl[d] == pytest.approx((lp - lm) / (2 * h), rel=2e-4, abs=1e-6)
