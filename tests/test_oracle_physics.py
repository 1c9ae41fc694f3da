"""Pins of the oracle's physics: entropy variables, log mean, EC flux, Roe dissipation."""
import mpmath
import numpy as np
import pytest

from oracle import physics

G = 1.4


def random_states(n, seed, spread=0.5):
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(-spread, spread, n))
    vel = rng.uniform(-1, 1, (3, n))
    p = np.exp(rng.uniform(-spread, spread, n)) * 2.0
    rho_e = p / (G - 1) + 0.5 * rho * np.sum(vel * vel, axis=0)
    return np.concatenate([rho[None], rho * vel, rho_e[None]])


def test_entropy_variables_round_trip():
    U = random_states(10000, 1)
    V = physics.entropy_variables(U, G)
    U2 = physics.conserved_from_entropy(V, G)
    assert np.max(np.abs(U2 - U) / np.abs(U).max(axis=0)) < 2e-14


def test_entropy_variables_are_gradient_of_entropy():
    """v = dU/du, checked by the complex-step derivative of U(u)."""
    U = random_states(200, 2)
    V = physics.entropy_variables(U, G)
    h = 1e-30
    for k in range(5):
        Uc = U.astype(complex)
        Uc[k] += 1j * h
        dS = np.imag(physics.entropy_function(Uc, G)) / h
        assert np.allclose(dS, V[k], rtol=1e-13, atol=1e-13)


def test_entropy_potential_identity():
    """psi = v . f - F with entropy flux F = U u (Eq. entropy pot with flux relationship)."""
    U = random_states(500, 3)
    rng = np.random.default_rng(4)
    nvec = rng.standard_normal((3, 500))
    V = physics.entropy_variables(U, G)
    f = physics.euler_flux(U, nvec, G)
    rho, vel, p = physics.primitive(U, G)
    Fent = physics.entropy_function(U, G) * np.sum(vel * nvec, axis=0)
    assert np.allclose(np.sum(V * f, axis=0) - Fent, physics.entropy_potential(U, nvec), rtol=1e-12, atol=1e-12)


def test_log_mean_against_extended_precision():
    rng = np.random.default_rng(5)
    a = np.exp(rng.uniform(-3, 3, 3000))
    ratio = np.concatenate([1 + rng.uniform(-1e-2, 1e-2, 1000), 1 + rng.uniform(-0.3, 0.3, 1000),
                            np.exp(rng.uniform(-3, 3, 1000))])
    b = a * ratio
    lm = physics.log_mean(a, b)
    mpmath.mp.dps = 40
    worst = 0.0
    for ai, bi, li in zip(a, b, lm):
        A, B = mpmath.mpf(float(ai)), mpmath.mpf(float(bi))
        ref = A if A == B else (A - B) / (mpmath.log(A) - mpmath.log(B))
        worst = max(worst, abs(float((mpmath.mpf(float(li)) - ref) / ref)))
    assert worst < 2e-15
    assert np.array_equal(physics.log_mean(a, a), a)


def test_chandrashekar_consistency_and_symmetry():
    U = random_states(2000, 6)
    rng = np.random.default_rng(7)
    nvec = rng.standard_normal((3, 2000))
    F = physics.chandrashekar(U, U, nvec, G)
    f = physics.euler_flux(U, nvec, G)
    assert np.allclose(F, f, rtol=1e-14, atol=1e-14 * np.abs(f).max())
    U2 = random_states(2000, 8)
    assert np.allclose(physics.chandrashekar(U, U2, nvec, G), physics.chandrashekar(U2, U, nvec, G),
                       rtol=1e-14, atol=1e-14)


def _linearity_defect(F):
    """max over variables of |F(l n1 + m n2) - l F(n1) - m F(n2)| / scale on random pairs."""
    U, U2 = random_states(1000, 21), random_states(1000, 22)
    rng = np.random.default_rng(23)
    n1, n2 = rng.standard_normal((3, 1000)), rng.standard_normal((3, 1000))
    lam, mu = rng.uniform(-3, 3, 1000), rng.uniform(-3, 3, 1000)
    lhs = F(U, U2, lam * n1 + mu * n2, G)
    rhs = lam * F(U, U2, n1, G) + mu * F(U, U2, n2, G)
    scale = np.abs(lam * F(U, U2, n1, G)).max(axis=1, keepdims=True) + np.abs(mu * F(U, U2, n2, G)).max(
        axis=1, keepdims=True)
    return float((np.abs(lhs - rhs) / scale).max())


@pytest.mark.parametrize("flux", ["chandrashekar", "ranocha"])
def test_two_point_fluxes_are_linear_in_the_metric_row(flux):
    """F(u_a, u_b; l n1 + m n2) = l F(n1) + m F(n2): the volume kernels rely on it to average
    the two nodes' metric rows once per pair and to fold the pair's weight in the Hadamard sum
    (S1_ab, or t_s,a for a hybrid pair; Eq. NSFR) into that row, signs included."""
    assert _linearity_defect(getattr(physics, flux)) <= 1e-14


def test_linearity_pin_catches_a_unit_normal_pressure_term():
    """A pressure term taken along the unit normal (p_hat n/|n| in place of p_hat n) keeps the
    flux consistent for unit rows but breaks linearity, and the pin above sees it."""
    def planted(UL, UR, nvec, gamma):
        F = physics.chandrashekar(UL, UR, nvec, gamma)
        nn = np.sqrt(np.sum(nvec * nvec, axis=0))
        p_hat = physics.chandrashekar(UL, UR, np.array([[1.0], [0.0], [0.0]]) * np.ones_like(nvec[:1]), gamma)
        # p_hat from the x-momentum flux along e_x minus its convective part
        rl, ul, _ = physics.primitive(UL, gamma)
        rr, ur, _ = physics.primitive(UR, gamma)
        ubar = 0.5 * (ul + ur)
        p_hat = p_hat[1] - p_hat[0] * ubar[0]
        F[1:4] += p_hat * nvec * (1.0 / nn - 1.0)
        return F
    assert _linearity_defect(planted) > 1e-3


@pytest.mark.parametrize("spread", [1e-3, 0.05, 0.8])
def test_tadmor_shuffle(spread):
    """[[v]] . f_s . n = [[psi . n]] for every pair (Eq. Tadmor shuffle quad node)."""
    n = 100000
    UL = random_states(n, 9, 0.5)
    rng = np.random.default_rng(10)
    rhoR = UL[0] * np.exp(rng.uniform(-spread, spread, n))
    rL, uL, pL = physics.primitive(UL, G)
    uR = uL + rng.uniform(-spread, spread, (3, n))
    pR = pL * np.exp(rng.uniform(-spread, spread, n))
    UR = np.concatenate([rhoR[None], rhoR * uR, (pR / (G - 1) + 0.5 * rhoR * np.sum(uR * uR, axis=0))[None]])
    nvec = rng.standard_normal((3, n))
    F = physics.chandrashekar(UL, UR, nvec, G)
    dv = physics.entropy_variables(UL, G) - physics.entropy_variables(UR, G)
    lhs = np.sum(dv * F, axis=0)
    rhs = physics.entropy_potential(UL, nvec) - physics.entropy_potential(UR, nvec)
    # rounding scale of both sides: the jumps are formed from O(|v|) values
    vabs = np.abs(physics.entropy_variables(UL, G)) + np.abs(physics.entropy_variables(UR, G))
    scale = np.sum(vabs * np.abs(F), axis=0) + np.abs(physics.entropy_potential(UL, nvec)) \
        + np.abs(physics.entropy_potential(UR, nvec))
    assert np.max(np.abs(lhs - rhs) / scale) < 2e-15


def test_shuffle_fails_for_a_wrong_energy_flux(monkeypatch):
    """Planted mistake: replacing |u|^2_bar by |u_bar|^2 must break the shuffle pin."""
    n = 2000
    UL, UR = random_states(n, 11), random_states(n, 12)
    nvec = np.random.default_rng(13).standard_normal((3, n))

    def wrong(UL, UR, nvec, gamma):
        F = physics.chandrashekar(UL, UR, nvec, gamma)
        _, uL, _ = physics.primitive(UL, gamma)
        _, uR, _ = physics.primitive(UR, gamma)
        ub = 0.5 * (uL + uR)
        q2 = 0.5 * (np.sum(uL * uL, 0) + np.sum(uR * uR, 0))
        F[4] += 0.5 * F[0] * (q2 - np.sum(ub * ub, 0))
        return F

    F = wrong(UL, UR, nvec, G)
    dv = physics.entropy_variables(UL, G) - physics.entropy_variables(UR, G)
    err = np.sum(dv * F, 0) - (physics.entropy_potential(UL, nvec) - physics.entropy_potential(UR, nvec))
    assert np.max(np.abs(err)) > 1e-6


def test_roe_linearisation_property():
    """A_roe (u_R - u_L) = (f(u_R) - f(u_L)) . n: Roe's defining property."""
    n = 5000
    UL, UR = random_states(n, 14), random_states(n, 15)
    nvec = np.random.default_rng(16).standard_normal((3, n))
    A_du = physics.roe_matrix_apply(UL, UR, nvec, G, absolute=False)
    df = physics.euler_flux(UR, nvec, G) - physics.euler_flux(UL, nvec, G)
    assert np.allclose(A_du, df, rtol=1e-11, atol=1e-11 * np.abs(df).max())
    assert np.allclose(physics.roe_matrix_apply(UL, UL, nvec, G), 0.0, atol=1e-13)
    # |A| is positive semi-definite along the jump in entropy variables for small jumps
    UR2 = UL * (1 + 1e-4 * np.random.default_rng(17).standard_normal(UL.shape))
    dv = physics.entropy_variables(UR2, G) - physics.entropy_variables(UL, G)
    q = np.sum(dv * physics.roe_matrix_apply(UL, UR2, nvec, G), axis=0)
    assert np.all(q > -1e-14)
