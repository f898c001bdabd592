"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle on the CPU: a dropped factor, a wrong exponent, a
reversed order, a transposed operand, a sign, an off-by-one.  It then runs a pin from
test_oracle_pins.py and expects that pin to fail.  The mistakes are planted with monkeypatch,
so nothing outside the test changes.  A case that passed would mean the pins do not see that
mistake.
"""
import numpy as np
import pytest

import test_oracle_pins as P
from oracle import rs_oracle as O
from workloads import load_config, make_particles

ORIG = {name: getattr(O, name) for name in dir(O) if callable(getattr(O, name))}


def _c1():
    cfg = load_config("c1_box64_n129")
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    return pr, pr.Pl_grid()


def _small():
    rng = np.random.default_rng(21)
    xyz, z = P.random_particles(rng, 6, 3.0, 1.0)
    pr = O.Problem(P.small_cfg(), xyz, z)
    return pr, pr.Pl_grid()


def _matvec():
    rng = np.random.default_rng(3)
    cfg = P.small_cfg(b=2.0, n=11, R=10, R_s=3, h_q=0.8, u0=-4.0, delta_rel=1e-6)
    xyz, z = P.random_particles(rng, 6, 1.8, 0.7)
    pr = O.Problem(cfg, xyz, z)
    return pr, O.rs_matrix_dense(pr.pk, pr.klong, pr.kshort, pr.gamma, pr.n)


# -- planted mistakes ---------------------------------------------------------------------------
def cell_integral_not_average(t, h, c):
    """Eq. (2.5) without the 1/h of the cell average."""
    return ORIG["cell_average_gaussian"](t, h, c) * h


def quadrature_without_step(R, h_q, u0):
    """Sinc weights a_k without the step h_q."""
    t, a = ORIG["sinc_quadrature"](R, h_q, u0)
    return t, a / h_q


def split_reversed(R, R_s):
    """Long part = the largest t_k (the split of Eq. (2.11) read the wrong way round)."""
    return np.arange(R_s, R), np.arange(R_s)


def gamma_one_short(pk, kshort, n, delta):
    """Window half-width one step short of criterion (A)."""
    return max(0, ORIG["window_halfwidth"](pk, kshort, n, delta) - 1)


def side_weight_square_root(j, z, pk, klong, n):
    """Column weights |z|^{1/2} instead of |z|^{1/3}."""
    Us, xi = ORIG["side_matrices"](j, z, pk, klong, n)
    f = np.repeat(np.abs(np.asarray(z, float)) ** (1.0 / 6.0), len(klong))
    return [U * f[None, :] for U in Us], xi


def rank_rule_without_third(sigma, eps, cap=0):
    """Tail budget eps^2 instead of eps^2/3 per mode."""
    return ORIG["rhosvd_rank"](sigma, eps * np.sqrt(3.0), cap)


def rhosvd_core_transposed(Us, xi, eps, cap=0, ranks=None):
    """Core with its last two indices swapped."""
    Z0s, beta, rk, sig = ORIG["rhosvd"](Us, xi, eps, cap, ranks)
    return Z0s, np.ascontiguousarray(beta.transpose(0, 2, 1)), rk, sig


def mode_matrix_without_signs(Us, xi, Vs, l):
    """M_{U_l} with the weights xi replaced by their magnitudes."""
    return ORIG["als_mode_matrix"](Us, np.abs(xi), Vs, l)


def als_core_from_start_bases(Us, xi, Z0s, eps, cap=0, sweeps=1, ranks=None):
    """Step (V) projected onto the starting bases instead of the final ones."""
    Vs, beta, rk = ORIG["c2t_als"](Us, xi, Z0s, eps, cap, sweeps, ranks)
    Z0 = [np.asarray(Z)[:, : V.shape[1]] for Z, V in zip(Z0s, Vs)]
    Y = [Z0[l].T @ Us[l] for l in range(3)]
    return Vs, np.einsum("aK,bK,cK,K->abc", Y[0], Y[1], Y[2], xi, optimize=True), rk


def als_jacobi_order(Us, xi, Z0s, eps, cap=0, sweeps=1, ranks=None):
    """Every mode of a sweep updated from the previous sweep's bases (not in order)."""
    Vs = [np.asarray(Z, float) for Z in Z0s]
    rk = [V.shape[1] for V in Vs]
    for _ in range(int(sweeps)):
        new = []
        for l in range(3):
            Zl, s, _ = np.linalg.svd(ORIG["als_mode_matrix"](Us, xi, Vs, l), full_matrices=False)
            r = ORIG["rhosvd_rank"](s, eps, cap) if ranks is None else int(ranks[l])
            new.append(Zl[:, :r])
            rk[l] = r
        Vs = new
    Y = [Vs[l].T @ Us[l] for l in range(3)]
    return Vs, np.einsum("aK,bK,cK,K->abc", Y[0], Y[1], Y[2], xi, optimize=True), rk


def energy_without_half(p_at_particles, z, self_value):
    """Eq. (4.7) without the factor 1/2."""
    return 2.0 * ORIG["energy_from_potential"](p_at_particles, z, self_value)


def forces_wrong_sign(xyz, z):
    """F = +dE/dx."""
    return -ORIG["forces_direct"](xyz, z)


def fd_matrix_transposed(n, h, order=8):
    """The difference operator applied as D_h^T (rows and columns exchanged)."""
    return ORIG["fd_matrix"](n, h, order).T.copy()


def tucker_fd_wrong_mode(j, z, pk, dpk, klong, kshort, gamma, Z0s, beta, D):
    """The mode-1 derivative taken along mode 2 (the difference of the wrong basis)."""
    F = ORIG["rs_tucker_fd_forces"](j, z, pk, dpk, klong, kshort, gamma, Z0s, beta, D)
    G = ORIG["rs_tucker_fd_forces"](j, z, pk, dpk, klong, kshort, gamma, [Z0s[1], Z0s[0], Z0s[2]],
                                    beta.transpose(1, 0, 2), D)
    F[:, 0] = G[:, 1]
    return F


def rs_matrix_short_uncut(pk, klong, kshort, gamma, n):
    """The short-range terms of the RS matrix without their window."""
    return ORIG["rs_matrix_dense"](pk, klong, kshort, n, n)


def energy_matvec_with_diagonal(pk, klong, kshort, gamma, n, j, z):
    """1/2 <A z, z> with the diagonal (self-interaction) left in."""
    C = ORIG["charge_grid"](j, z, n)
    return ORIG["energy_matvec"](pk, klong, kshort, gamma, n, j, z) + 0.5 * float(
        np.sum(C * C)) * float(np.sum(pk[:, n - 1] ** 3))


def snap_half_to_even(xyz, b, h, n):
    """Ties rounded half to even instead of away from zero."""
    j = np.rint((np.asarray(xyz, float) + b) / h).astype(np.int64)
    if np.any(j < 0) or np.any(j >= n):
        raise ValueError("centre outside the box")
    return j


CASES = [
    ("cell_average_gaussian", cell_integral_not_average,
     lambda: P.test_cell_average_matches_numerical_integration(0.7, 0.15625)),
    ("sinc_quadrature", quadrature_without_step, lambda: P.test_quadrature_approximates_inverse_distance("c1_box64_n129")),
    ("split", split_reversed, P.test_split_identity_and_order),
    ("window_halfwidth", gamma_one_short, P.test_window_truncation_and_minimal_gamma),
    ("side_matrices", side_weight_square_root, lambda: P.test_side_matrices_reproduce_long_range_sum(_c1())),
    ("rhosvd_rank", rank_rule_without_third, lambda: P.test_rhosvd_rank_rule_and_cap(_c1())),
    ("rhosvd", rhosvd_core_transposed, lambda: P.test_rhosvd_error_within_eps_and_pythagoras(_c1(), 1e-4)),
    ("als_mode_matrix", mode_matrix_without_signs, lambda: P.test_als_mode_matrix_is_the_projected_dense_unfolding(_small())),
    ("c2t_als", als_core_from_start_bases, lambda: P.test_als_matches_dense_hooi(_small(), False)),
    ("c2t_als", als_jacobi_order, lambda: P.test_als_matches_dense_hooi(_small(), True)),
    ("energy_from_potential", energy_without_half, P.test_energy_tensor_formula_matches_direct),
    ("forces_direct", forces_wrong_sign, P.test_forces_direct_finite_difference),
    ("snap_to_grid", snap_half_to_even, P.test_snap_rounding_and_bounds),
    ("rs_matrix_dense", rs_matrix_short_uncut,
     lambda: P.test_rs_matvec_of_the_charges_is_the_rs_canonical_tensor(_matvec())),
    ("energy_matvec", energy_matvec_with_diagonal, lambda: P.test_energy_through_the_matrix(_matvec())),
    ("fd_matrix", fd_matrix_transposed, lambda: P.test_fd_forces_converge_to_the_analytic_long_range_forces(_c1())),
    ("rs_tucker_fd_forces", tucker_fd_wrong_mode,
     lambda: P.test_tucker_fd_forces_exact_at_full_rank_and_within_eps(_c1())),
]


@pytest.mark.parametrize("name,mutant,pin", CASES, ids=[f"{c[0]}-{c[1].__name__}" for c in CASES])
def test_pin_catches_planted_mistake(monkeypatch, name, mutant, pin):
    monkeypatch.setattr(O, name, mutant)
    with pytest.raises(AssertionError):
        pin()


def test_pins_pass_without_mistakes():
    """The same pin calls pass on the unmodified oracle (so the failures above are the planted
    mistakes, not the way the pins are called)."""
    for _, _, pin in CASES:
        pin()
