"""Pins for the tetrahedron oracle: rest stability, the linear-elastic small-strain limit,
rotation invariance, finite differences, PSD projection, lumped mass."""
import numpy as np
import pytest

from oracle import tet as O

E, NU = 1e5, 0.4
MU, LAM = O.snh_params(E, NU)


def _rand_tet(rng, scale=0.1, jitter=0.2):
    base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * scale
    return base + rng.normal(scale=jitter * scale, size=(4, 3)) + rng.uniform(0, 1, 3)


def _commutation():
    K = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            K[i + 3 * j, j + 3 * i] = 1.0
    return K


def test_rest_is_stress_free():
    _, g, _ = O.psi_derivs(np.eye(3), MU, LAM)
    assert np.abs(g).max() <= 1e-10 * MU


def test_small_strain_limit_is_linear_elasticity():
    """d2Psi/dF2 at F = I equals mu_L (I + K) + lam_L vec(I) vec(I)^T."""
    mu_l, lam_l = O.lame(E, NU)
    _, _, H = O.psi_derivs(np.eye(3), MU, LAM)
    vI = np.eye(3).reshape(-1, order="F")
    C = mu_l * (np.eye(9) + _commutation()) + lam_l * np.outer(vI, vI)
    np.testing.assert_allclose(H, C, rtol=1e-12, atol=1e-9 * mu_l)


def test_energy_derivatives_match_finite_differences():
    rng = np.random.default_rng(1)
    F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    e, g, H = O.psi_derivs(F, MU, LAM)
    h = 1e-6
    for k in range(9):
        dF = np.zeros(9)
        dF[k] = h
        fp = O.psi_derivs(F + dF.reshape(3, 3, order="F"), MU, LAM)
        fm = O.psi_derivs(F - dF.reshape(3, 3, order="F"), MU, LAM)
        assert (fp[0] - fm[0]) / (2 * h) == pytest.approx(g[k], rel=1e-6, abs=1e-6 * MU)
        np.testing.assert_allclose((fp[1] - fm[1]) / (2 * h), H[:, k], rtol=1e-5, atol=1e-5 * MU)


def test_deformation_gradient_map_is_exact():
    rng = np.random.default_rng(2)
    rest = _rand_tet(rng)
    Dmi, _ = O.rest_shape(rest)
    D = O.dF_dx(Dmi)
    P = rest + 0.02 * rng.normal(size=(4, 3))
    Ds = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)
    np.testing.assert_allclose(D @ P.reshape(-1), (Ds @ Dmi).reshape(-1, order="F"), rtol=1e-13, atol=1e-13)


def test_rotation_invariance():
    rng = np.random.default_rng(3)
    rest = _rand_tet(rng)
    Dmi, vol = O.rest_shape(rest)
    P = rest + 0.02 * rng.normal(size=(4, 3))
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)], [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                  [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])
    r0 = O.eval_tet(P, Dmi, vol, MU, LAM, 1e-4)
    r1 = O.eval_tet(P @ R.T, Dmi, vol, MU, LAM, 1e-4)
    Rb = np.kron(np.eye(4), R)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["grad"], Rb @ r0["grad"], rtol=1e-10, atol=1e-12 * np.abs(r0["grad"]).max())
    np.testing.assert_allclose(r1["hess"], Rb @ r0["hess"] @ Rb.T, rtol=1e-9, atol=1e-11 * np.abs(r0["hess"]).max())


def test_gradient_and_hessian_against_fd_in_positions():
    """Gradient and the unprojected x-space Hessian D^T (d2Psi/dF2) D against finite differences.
    (Near rest the twist eigenvalues are ~0 and may be slightly negative, so the projected block
    is compared separately: it is the PSD part of this matrix in F-space.)"""
    rng = np.random.default_rng(4)
    rest = _rand_tet(rng)
    Dmi, vol = O.rest_shape(rest)
    P = rest + 0.01 * rng.normal(size=(4, 3))
    r = O.eval_tet(P, Dmi, vol, MU, LAM, 1.0)
    D = O.dF_dx(Dmi)
    _, _, H9 = O.psi_derivs(r["F"], MU, LAM)
    Hx = vol * D.T @ H9 @ D
    h = 1e-7
    for idx in range(12):
        Pp, Pm = P.copy(), P.copy()
        Pp[idx // 3, idx % 3] += h
        Pm[idx // 3, idx % 3] -= h
        rp, rm = O.eval_tet(Pp, Dmi, vol, MU, LAM, 1.0), O.eval_tet(Pm, Dmi, vol, MU, LAM, 1.0)
        assert (rp["energy"] - rm["energy"]) / (2 * h) == pytest.approx(r["grad"][idx], rel=1e-5,
                                                                        abs=1e-6 * np.abs(r["grad"]).max())
        np.testing.assert_allclose((rp["grad"] - rm["grad"]) / (2 * h), Hx[:, idx], rtol=1e-4,
                                   atol=1e-5 * np.abs(Hx).max())
    np.testing.assert_allclose(r["hess"], vol * D.T @ O.project_psd(H9) @ D, rtol=1e-12,
                               atol=1e-12 * np.abs(Hx).max())


def test_projection_is_psd_even_when_inverted():
    rng = np.random.default_rng(5)
    rest = _rand_tet(rng)
    Dmi, vol = O.rest_shape(rest)
    P = rest.copy()
    P[3] = P[0] - (P[3] - P[0]) * 0.5           # flip the fourth vertex through the base
    r = O.eval_tet(P, Dmi, vol, MU, LAM, 1.0)
    assert np.linalg.det(r["F"]) < 0
    ev = np.linalg.eigvalsh(r["hess"])
    assert ev.min() >= -1e-9 * ev.max()
    _, _, H9 = O.psi_derivs(r["F"], MU, LAM)
    assert np.linalg.eigvalsh(H9).min() < 0     # the exact Hessian is indefinite there


def test_lumped_mass_sums_to_total_mass():
    rng = np.random.default_rng(6)
    n, T = 30, 40
    x = rng.uniform(0, 1, (3, n))
    tets = np.stack([rng.choice(n, 4, replace=False) for _ in range(T)], 1)
    Dmi, vol, mass = O.rest_state(x, tets, 1000.0)
    assert mass.sum() == pytest.approx(1000.0 * vol.sum(), rel=1e-13)
    for t in range(T):
        inv = Dmi[:, t].reshape(3, 3)
        P = x[:, tets[:, t]].T
        Dm = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)
        np.testing.assert_allclose(inv @ Dm, np.eye(3), atol=1e-9)
