"""Pins of the CPU oracle against facts that do not come from the oracle itself:
numerical integration, closed forms, brute force on tiny grids, invariants and
textbook constants.  Each test names the passage it pins; a plausible mistake in
the oracle (dropped term, wrong sign, transposed operand, wrong normalisation)
fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import rs_oracle as O
from workloads import load_config, make_particles

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def small_cfg(**kw):
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8)
    cfg.update(kw)
    return cfg


def random_particles(rng, N, half, sep):
    pts = []
    while len(pts) < N:
        x = rng.uniform(-half, half, 3)
        if all(np.linalg.norm(x - p) >= sep for p in pts):
            pts.append(x)
    return np.array(pts), rng.uniform(-1, 1, N)


# ---------------------------------------------------------------- Sec. 2.2 factors
@pytest.mark.parametrize("t", [1e-4, 0.03, 0.7, 3.0, 30.0])
@pytest.mark.parametrize("h", [0.03125, 0.15625])
def test_cell_average_matches_numerical_integration(t, h):
    """Galerkin factor (Eq. (2.5), vectors before Eq. (2.10)) against adaptive quadrature."""
    for d in [0, 1, 2, 5, 17, 60]:
        c = d * h
        ref, _ = integrate.quad(lambda x: math.exp(-t * t * x * x), c - h / 2, c + h / 2,
                                epsabs=0.0, epsrel=1e-13, limit=200)
        got = float(O.cell_average_gaussian(t, h, c)) * h
        if ref > 1e-250:
            assert abs(got - ref) <= 1e-11 * ref + 1e-300, (t, h, d, got, ref)
        # symmetric in the offset
        assert float(O.cell_average_gaussian(t, h, -c)) == float(O.cell_average_gaussian(t, h, c))


def test_cell_average_small_t_limit_and_total_mass():
    """t -> 0: the cell average of exp(-t^2 x^2) tends to 1; summing the cell integrals
    over all cells gives int_R exp(-t^2 x^2) dx = sqrt(pi)/t (golden closed form)."""
    assert abs(float(O.cell_average_gaussian(1e-9, 0.1, 0.0)) - 1.0) < 1e-15
    g = GOLD["gaussian_integral"]
    h = 0.05
    d = np.arange(-4000, 4001) * h
    total = float(np.sum(O.cell_average_gaussian(g["t"], h, d)) * h)
    assert abs(total - g["value"]) < 1e-12 * g["value"]


def test_reference_factors_layout_and_weights():
    """p_k[d] = a_k^{1/3} * cell average (Eq. (2.10)); stored at column d + n - 1."""
    t, a = O.sinc_quadrature(6, 0.8, -3.0)
    h, n = 0.1, 9
    pk = O.reference_factors(t, a, h, n)
    assert pk.shape == (6, 2 * n - 1)
    for k in range(6):
        for d in (-8, -3, 0, 4, 8):
            ref, _ = integrate.quad(lambda x: math.exp(-t[k] ** 2 * x * x), d * h - h / 2, d * h + h / 2,
                                    epsabs=0, epsrel=1e-13)
            assert abs(pk[k, d + n - 1] - a[k] ** (1 / 3) * ref / h) <= 1e-11 * abs(pk[k, d + n - 1])


# ---------------------------------------------------------------- Sec. 2.2 quadrature
@pytest.mark.parametrize("name", ["c1_box64_n129", "c2_protein1000_n513", "c3_nacl28_n1025", "c5_forces4096_n513"])
def test_quadrature_approximates_inverse_distance(name):
    """sum_k a_k exp(-t_k^2 rho^2) ~ 1/rho (Eqs. (2.6)-(2.8)) within the fitted error, on a
    radius grid denser than the one used by the fit."""
    cfg = load_config(name)
    t, a = O.sinc_quadrature(cfg["R"], cfg["h_q"], cfg["u0"])
    f = cfg["fit"]
    rho = np.geomspace(f["rho_min"], f["rho_max"], 20011)
    err = np.max(np.abs(O.kernel_sum(t, a, rho) * rho - 1.0))
    assert err <= f["max_rel_err"] * 1.02 + 1e-12
    assert err < 6e-3


def test_quadrature_converges_exponentially():
    """Eq. (2.9): the error decays like exp(-beta sqrt(M)); doubling R at a fixed range must
    cut the best error by orders of magnitude."""
    from scipy.optimize import minimize
    rho = np.geomspace(0.05, 30.0, 3000)

    def best(R):
        f = lambda p: np.max(np.abs(O.kernel_sum(*O.sinc_quadrature(R, p[0], p[1]), rho) * rho - 1))
        cands = [(f([hq, u]), hq, u) for hq in np.linspace(0.3, 1.5, 13) for u in np.linspace(-12, -2, 21)]
        _, hq, u = min(cands)
        return minimize(f, [hq, u], method="Nelder-Mead", options=dict(xatol=1e-9, fatol=1e-14, maxiter=4000)).fun

    e12, e24, e36 = best(12), best(24), best(36)
    assert e24 < 0.1 * e12 and e36 < 0.1 * e24


# ---------------------------------------------------------------- Sec. 3.2 canonical sum
def test_brute_force_tiny_grid():
    """P_0 entry by entry from the definition (Eqs. (2.5), (2.10), (3.4)): for every grid
    cell and particle, the cell average of each Gaussian integrated numerically in each
    coordinate; no closed form, no shifted arrays."""
    rng = np.random.default_rng(7)
    cfg = small_cfg(b=2.0, n=9, R=6, R_s=2, h_q=0.9, u0=-2.5)
    h, x = O.grid(cfg["b"], cfg["n"])
    t, a = O.sinc_quadrature(cfg["R"], cfg["h_q"], cfg["u0"])
    pk = O.reference_factors(t, a, h, cfg["n"])
    j = rng.integers(0, cfg["n"], (3, 3))
    z = np.array([0.7, -1.1, 0.4])
    P = O.canonical_sum_grid(j, z, pk, np.arange(cfg["R"]), cfg["n"])
    xc = x[j]                                   # centres
    n = cfg["n"]
    for i1 in range(n):
        for i2 in range(0, n, 2):
            for i3 in range(0, n, 3):
                s = 0.0
                for nu in range(3):
                    for k in range(cfg["R"]):
                        prod = a[k]
                        for l, il in enumerate((i1, i2, i3)):
                            lo, hi = x[il] - h / 2 - xc[nu, l], x[il] + h / 2 - xc[nu, l]
                            v, _ = integrate.quad(lambda y: math.exp(-t[k] ** 2 * y * y), lo, hi,
                                                  epsabs=0, epsrel=1e-12)
                            prod *= v / h
                        s += z[nu] * prod
                assert abs(P[i1, i2, i3] - s) <= 1e-10 * max(1.0, abs(s)), (i1, i2, i3)


def cube_average_direct(xyz_src, z, centre, h, q=6):
    """Average of sum_nu z_nu/|x - x_nu| over the cube of side h at ``centre``
    (tensor Gauss-Legendre rule); the closed-form counterpart of a Galerkin cell value."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = g * h / 2
    w = w / 2
    X = centre[None, None, None, :] + np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    tot = 0.0
    for nu in range(len(z)):
        r = np.linalg.norm(X - xyz_src[nu], axis=-1)
        tot += z[nu] * float(np.sum(W / r))
    return tot


def test_P0_matches_closed_form_inverse_distance():
    """P_0 (Eq. (3.4)) against the cell average of sum z/|x - x_nu| (Eq. (1.1)) at grid
    points at least 3h from every particle: the difference is bounded by the
    quadrature's relative error times sum |z|/r."""
    cfg = load_config("c1_box64_n129")
    parts = make_particles(cfg)
    pr = O.Problem(cfg, parts.xyz, parts.Z)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, pr.n, (400, 3))
    X = pr.x[idx]
    d = np.linalg.norm(X[:, None, :] - pr.xyz_snapped[None], axis=-1)
    ok = d.min(1) >= 3 * pr.h
    idx, X, d = idx[ok][:120], X[ok][:120], d[ok][:120]
    P = pr.P0_points(idx)
    qerr = cfg["fit"]["max_rel_err"] * 1.02
    for m in range(len(idx)):
        ref = cube_average_direct(pr.xyz_snapped, pr.z, X[m], pr.h)
        bound = qerr * float(np.sum(np.abs(pr.z) / d[m])) + 1e-9
        assert abs(P[m] - ref) <= bound, (m, P[m], ref, bound)


def test_points_and_grid_evaluations_agree():
    cfg = small_cfg()
    rng = np.random.default_rng(11)
    xyz, z = random_particles(rng, 5, 3.0, 1.0)
    pr = O.Problem(cfg, xyz, z)
    G = pr.P0_grid()
    idx = rng.integers(0, pr.n, (200, 3))
    assert np.allclose(pr.P0_points(idx), G[idx[:, 0], idx[:, 1], idx[:, 2]], rtol=1e-13, atol=1e-13)


def test_direct_sum_golden_point():
    xyz = np.array([[0.0, 0, 0], [3.0, 4.0, 0]])
    z = np.array([2.0, -5.0])
    v = O.direct_sum_points(xyz, z, np.array([[0.0, 0.0, 1.0]]))[0]
    assert abs(v - (2.0 / 1.0 - 5.0 / math.sqrt(26.0))) < 1e-15


# ---------------------------------------------------------------- Sec. 2.3 split, Sec. 3.3 windows
def test_split_identity_and_order():
    """P_R = P_{R_s} + P_{R_l} (Eq. (2.12)); the long part holds the smallest t_k."""
    cfg = small_cfg()
    rng = np.random.default_rng(5)
    xyz, z = random_particles(rng, 6, 3.0, 1.0)
    pr = O.Problem(cfg, xyz, z)
    assert len(pr.klong) == cfg["R"] - cfg["R_s"] and len(pr.kshort) == cfg["R_s"]
    assert pr.t[pr.klong].max() < pr.t[pr.kshort].min()
    P0, Pl, Ps = pr.P0_grid(), pr.Pl_grid(), pr.Ps_grid()
    assert np.max(np.abs(Pl + Ps - P0)) <= 1e-13 * np.max(np.abs(P0))


def test_window_truncation_and_minimal_gamma():
    """Windows (Def. 3.4, Def. 3.6) hold the short-range part up to the cut-off: each
    particle loses at most delta*|z| at any point; gamma is the smallest such width."""
    cfg = small_cfg(n=41, delta_rel=1e-6)
    rng = np.random.default_rng(9)
    xyz, z = random_particles(rng, 4, 3.0, 1.5)
    pr = O.Problem(cfg, xyz, z)
    W, Ps = pr.windows_grid(), pr.Ps_grid()
    assert np.max(np.abs(W - Ps)) <= pr.delta * np.sum(np.abs(z)) * (1 + 1e-12)
    c = pr.n - 1
    g = pr.gamma
    assert np.sum(pr.pk[pr.kshort, c + g + 1] * pr.pk[pr.kshort, c] ** 2) <= pr.delta
    if g > 0:
        assert np.sum(pr.pk[pr.kshort, c + g] * pr.pk[pr.kshort, c] ** 2) > pr.delta
    # point evaluation of the windows matches the grid
    idx = rng.integers(0, pr.n, (300, 3))
    assert np.allclose(pr.windows_points(idx), W[idx[:, 0], idx[:, 1], idx[:, 2]], rtol=1e-13, atol=1e-15)


def test_block_orthogonality_of_disjoint_windows():
    """Prop. 3.11 (B), (C): windows with disjoint supports are orthogonal and their norms add."""
    cfg = small_cfg(n=41, delta_rel=1e-4)
    pr = O.Problem(cfg, np.array([[-2.5, -2.5, -2.5], [2.5, 2.5, 2.5]]), np.array([1.0, 1.0]))
    assert 2 * pr.gamma + 1 < abs(pr.j[0, 0] - pr.j[1, 0])
    U1 = O.windows_full(pr.j[:1], pr.z[:1], pr.pk, pr.kshort, pr.gamma, pr.n)
    U2 = O.windows_full(pr.j[1:], pr.z[1:], pr.pk, pr.kshort, pr.gamma, pr.n)
    assert float(np.sum(U1 * U2)) == 0.0
    U = pr.windows_grid()
    assert abs(np.sum(U * U) - np.sum(U1 * U1) - np.sum(U2 * U2)) <= 1e-12 * np.sum(U * U)


# ---------------------------------------------------------------- Sec. 6 RHOSVD
@pytest.fixture(scope="module")
def c1_problem():
    cfg = load_config("c1_box64_n129")
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    return pr, pr.Pl_grid()


def test_side_matrices_reproduce_long_range_sum(c1_problem):
    """xi x_l U^(l) (Eq. (2.4)) equals the long-range sum of Eq. (3.5) on the grid, and the
    canonical norm formula gives ||P_l||_F."""
    pr, Pl = c1_problem
    Us, xi = O.side_matrices(pr.j, pr.z, pr.pk, pr.klong, pr.n)
    P = np.einsum("iK,jK,kK,K->ijk", Us[0], Us[1], Us[2], xi, optimize=True)
    assert np.max(np.abs(P - Pl)) <= 1e-12 * np.max(np.abs(Pl))
    assert abs(O.canonical_norm2(Us, xi) - np.sum(Pl * Pl)) <= 1e-10 * np.sum(Pl * Pl)


def test_rhosvd_full_rank_is_exact(c1_problem):
    """Def. 6.1 with r_l = n keeps the whole column space: the projection is the identity."""
    pr, Pl = c1_problem
    Z0s, beta, rk, _, _, _ = pr.tucker(ranks=[pr.n] * 3)
    assert np.max(np.abs(O.tucker_full(beta, Z0s) - Pl)) <= 1e-11 * np.max(np.abs(Pl))


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_rhosvd_error_within_eps_and_pythagoras(c1_problem, eps):
    """RHOSVD Tucker error ||P_l - P_l^T||_F <= eps ||P_l||_F (Sec. 6, eps-truncation) on the
    full grid; the orthogonal projection obeys ||P_l||^2 = ||beta||^2 + ||P_l - P_l^T||^2."""
    pr, Pl = c1_problem
    Z0s, beta, rk, sig, _, _ = pr.tucker(eps=eps, cap=0)
    PT = O.tucker_full(beta, Z0s)
    nrm = np.linalg.norm(Pl)
    err = np.linalg.norm(Pl - PT)
    assert err <= eps * nrm
    assert abs(nrm ** 2 - np.sum(beta * beta) - err ** 2) <= 1e-9 * nrm ** 2
    for Z in Z0s:
        assert np.allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-12)


def test_rhosvd_rank_rule_and_cap(c1_problem):
    pr, _ = c1_problem
    _, _, rk, sig, _, _ = pr.tucker(eps=1e-6, cap=0)
    for l in range(3):
        e2 = sig[l] ** 2
        r = rk[l]
        assert e2[r:].sum() <= (1e-12 / 3) * e2.sum()
        assert e2[r - 1:].sum() > (1e-12 / 3) * e2.sum()
    _, beta, rk2, _, _, _ = pr.tucker(eps=1e-6, cap=16)
    assert max(rk2) <= 16 and beta.shape == tuple(rk2)


def test_rhosvd_bound_lemma(c1_problem):
    """Lemma 3.12 / the RHOSVD estimate: the Tucker error is controlled by the discarded
    side-matrix singular values, err <= sum_l (sum_{k>r_l} sigma_{l,k}^2)^{1/2} * ||xi||_inf-scaled
    (checked in the weaker relative form err/||P_l|| <= C sum_l tail_l/||U_l||_F with C = 10)."""
    pr, Pl = c1_problem
    Z0s, beta, rk, sig, Us, xi = pr.tucker(eps=1e-5, cap=0)
    err = np.linalg.norm(Pl - O.tucker_full(beta, Z0s)) / np.linalg.norm(Pl)
    rel_tails = sum(math.sqrt(np.sum(s[r:] ** 2) / np.sum(s ** 2)) for s, r in zip(sig, rk))
    assert err <= 10.0 * rel_tails


def test_tucker_rank_nearly_independent_of_N():
    """Theorem 3.2: the eps-rank of the long-range part depends on N only weakly."""
    cfg = load_config("c1_box64_n129")
    ranks = []
    for N in (16, 64, 160):
        c = dict(cfg)
        c["particles"] = dict(cfg["particles"], N=N)
        p = make_particles(c, seed=123 + N)
        pr = O.Problem(c, p.xyz, p.Z)
        _, _, rk, _, _, _ = pr.tucker(eps=1e-5, cap=0)
        ranks.append(max(rk))
    assert ranks[2] <= ranks[0] * 1.35 + 2, ranks


# ---------------------------------------------------------------- symmetries
def test_mirror_permutation_translation_linearity():
    """P_R has identical factors in the three modes (Sec. 2.2) and the kernel is radial:
    reflecting the particles in an axis reflects P_0, permuting axes permutes it, shifting
    by whole cells shifts it, and P_0 is linear in the charges."""
    cfg = small_cfg()
    rng = np.random.default_rng(21)
    xyz, z = random_particles(rng, 5, 2.5, 1.0)
    pr = O.Problem(cfg, xyz, z)
    P = pr.P0_grid()
    n = pr.n
    jr = pr.j.copy()
    jr[:, 0] = n - 1 - jr[:, 0]
    Pr = O.canonical_sum_grid(jr, z, pr.pk, pr.kall, n)
    assert np.allclose(Pr, P[::-1], rtol=1e-12, atol=1e-13)
    jp = pr.j[:, [2, 0, 1]]
    Pp = O.canonical_sum_grid(jp, z, pr.pk, pr.kall, n)
    assert np.allclose(Pp, P.transpose(2, 0, 1), rtol=1e-12, atol=1e-13)
    js = pr.j + np.array([2, -1, 3])
    Ps = O.canonical_sum_grid(js, z, pr.pk, pr.kall, n)
    assert np.allclose(Ps[2:, :-1, 3:], P[:-2, 1:, :-3], rtol=1e-12, atol=1e-13)
    P2 = O.canonical_sum_grid(pr.j, 2.5 * z, pr.pk, pr.kall, n)
    assert np.allclose(P2, 2.5 * P, rtol=1e-13, atol=1e-13)


def test_rs_tucker_mirror_symmetry(c1_problem):
    """The RS-Tucker approximation commutes with reflecting the particle set."""
    pr, _ = c1_problem
    Z0s, beta, rk, _, _, _ = pr.tucker(eps=1e-6, cap=0)
    P = O.tucker_full(beta, Z0s) + pr.windows_grid()
    xyz = pr.xyz.copy()
    xyz[:, 1] *= -1
    q = O.Problem(pr.cfg, xyz, pr.z)
    Z0q, bq, rq, _, _, _ = q.tucker(eps=1e-6, cap=0, ranks=rk)
    Q = O.tucker_full(bq, Z0q) + q.windows_grid()
    assert np.max(np.abs(Q - P[:, ::-1, :])) <= 1e-9 * np.max(np.abs(P))


def test_snap_rounding_and_bounds():
    h, x = O.grid(1.0, 5)   # h = 0.5
    j = O.snap_to_grid(np.array([[-1.0, 0.24, 0.25], [1.0, -0.25, 0.74]]), 1.0, h, 5)
    assert j.tolist() == [[0, 2, 3], [4, 2, 3]]
    with pytest.raises(ValueError):
        O.snap_to_grid(np.array([[1.2, 0, 0]]), 1.0, h, 5)


# ---------------------------------------------------------------- Sec. 4.2 energy, Sec. 4.3 forces
def test_energy_golden():
    for key in ("two_charge_energy", "three_charge_energy"):
        g = GOLD[key]
        assert abs(O.energy_direct(np.array(g["xyz"]), np.array(g["z"])) - g["E"]) < 1e-14


def test_energy_madelung_rock_salt():
    """Alternating-charge cubes (Table 4.4 lattices): the energy per ion extrapolates in
    1/L to -M/2 with the rock-salt Madelung constant (a factor-2 slip in Eq. (4.4) fails)."""
    M = GOLD["madelung_rock_salt"]["M"]
    e = {}
    for L in (10, 16):
        idx = np.stack(np.meshgrid(*[np.arange(L)] * 3, indexing="ij"), -1).reshape(-1, 3)
        z = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
        e[L] = O.energy_direct(idx.astype(float), z) / len(z)
    A = (16 * e[16] - 10 * e[10]) / 6.0
    assert abs(A + M / 2) < 0.01 * M / 2, (e, A)


def test_energy_tensor_formula_matches_direct():
    """Eq. (4.7): 1/2 sum z_j (P_0(x_j) - z_j P_R(0)) reproduces Eq. (4.4) within the
    quadrature error (relative to sum |z_j z_k|/r_jk)."""
    cfg = load_config("c1_box64_n129")
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    E = pr.energy_direct_snapped()
    Et = pr.energy_P0()
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    assert abs(Et - E) <= 1.05 * cfg["fit"]["max_rel_err"] * scale


def test_energy_long_range_lemma():
    """Lemma 4.1: when no other particle lies inside a short-range window, Eq. (4.6) with
    P_l alone equals Eq. (4.7) with P_0 up to the window cut-off."""
    cfg = small_cfg(b=8.0, n=65, R=16, R_s=5, h_q=0.75, u0=-7.5)
    rng = np.random.default_rng(31)
    xyz, z = random_particles(rng, 6, 6.5, 5.0)
    pr = O.Problem(cfg, xyz, z)
    assert pr.gamma * pr.h < 5.0 - 2 * pr.h
    E0 = pr.energy_P0()
    El = O.energy_from_potential(pr.Pl_points(pr.j), pr.z, pr.PRl0)
    assert abs(E0 - El) <= 0.5 * np.sum(np.abs(z)) ** 2 * pr.delta


def test_forces_direct_finite_difference():
    """F_j = -dE/dx_j for Eq. (4.4) (Sec. 4.3 without the printed factor 1/2)."""
    rng = np.random.default_rng(41)
    xyz, z = random_particles(rng, 8, 3.0, 1.0)
    F = O.forces_direct(xyz, z)
    hfd = 1e-5
    for j in range(8):
        for l in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[j, l] += hfd
            xm[j, l] -= hfd
            fd = -(O.energy_direct(xp, z) - O.energy_direct(xm, z)) / (2 * hfd)
            assert abs(fd - F[j, l]) <= 1e-7 * max(1.0, abs(F[j, l]))


def test_gaussian_pair_forces_finite_difference_and_coulomb_limit():
    """Pair-sum form of the long-range energy (Eq. (4.6), collocated Gaussians) and its
    forces: central differences, and with all R terms the Coulomb forces within the
    quadrature error."""
    cfg = load_config("c5_forces4096_n513")
    t, a = O.sinc_quadrature(cfg["R"], cfg["h_q"], cfg["u0"])
    rng = np.random.default_rng(43)
    xyz, z = random_particles(rng, 10, 5.0, 1.0)
    kl, _ = O.split(cfg["R"], cfg["R_s"])
    F = O.gaussian_pair_forces(xyz, z, t, a, kl)
    hfd = 1e-5
    for j in (0, 3, 7):
        for l in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[j, l] += hfd
            xm[j, l] -= hfd
            fd = -(O.gaussian_pair_energy(xp, z, t, a, kl) - O.gaussian_pair_energy(xm, z, t, a, kl)) / (2 * hfd)
            assert abs(fd - F[j, l]) <= 1e-7 * max(1.0, np.abs(F).max())
    Fall = O.gaussian_pair_forces(xyz, z, t, a, np.arange(cfg["R"]))
    Fc = O.forces_direct(xyz, z)
    assert np.max(np.abs(Fall - Fc)) <= 0.05 * np.max(np.abs(Fc))
    Eall = O.gaussian_pair_energy(xyz, z, t, a, np.arange(cfg["R"]))
    assert abs(Eall - O.energy_direct(xyz, z)) <= 1.05 * cfg["fit"]["max_rel_err"] * O.energy_scale(xyz, z)


# ---------------------------------------------------------------- Sec. 4.3 adjoint forces
def test_galerkin_factors_on_grid_and_derivative():
    """The continuous Galerkin factors reproduce the grid factors at grid offsets (Eq. (2.10)),
    and their closed-form derivative matches central differences of the factors themselves."""
    cfg = small_cfg()
    pr = O.Problem(cfg, np.zeros((1, 3)), np.ones(1))
    d = np.arange(-(pr.n - 1), pr.n) * pr.h
    assert np.allclose(O.galerkin_factors_at(pr.t, pr.a, pr.h, d), pr.pk, rtol=1e-13, atol=1e-15)
    y = np.linspace(-2.0, 2.0, 41) + 0.0123
    hf = 1e-5
    fd = (O.galerkin_factors_at(pr.t, pr.a, pr.h, y + hf) - O.galerkin_factors_at(pr.t, pr.a, pr.h, y - hf)) / (2 * hf)
    g = O.galerkin_factors_at(pr.t, pr.a, pr.h, y, derivative=True)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(g))
    # odd in the offset: zero derivative at the cell centre
    assert np.all(O.reference_factor_derivatives(pr.t, pr.a, pr.h, pr.n)[:, pr.n - 1] == 0.0)


def test_galerkin_pair_forces_finite_difference_momentum_and_limit():
    """F = -grad E for the Galerkin pair energy (central differences), total force zero
    (each pair contributes equal and opposite forces), and as h -> 0 the cell averages tend to
    point values so the forces tend to the collocated Gaussian-sum pair forces."""
    cfg = small_cfg()
    rng = np.random.default_rng(31)
    xyz, z = random_particles(rng, 6, 2.5, 1.0)
    pr = O.Problem(cfg, xyz, z)
    F = O.galerkin_pair_forces(xyz, z, pr.t, pr.a, pr.kall, pr.h)
    hfd = 1e-5
    for jj in range(3):
        for l in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[jj, l] += hfd
            xm[jj, l] -= hfd
            fd = -(O.galerkin_pair_energy(xp, z, pr.t, pr.a, pr.kall, pr.h)
                   - O.galerkin_pair_energy(xm, z, pr.t, pr.a, pr.kall, pr.h)) / (2 * hfd)
            assert abs(F[jj, l] - fd) <= 1e-7 * np.abs(F).max()
    assert np.abs(F.sum(0)).max() <= 1e-12 * np.abs(F).max()
    Fh = O.galerkin_pair_forces(xyz, z, pr.t, pr.a, pr.kall, 1e-3)
    Fg = O.gaussian_pair_forces(xyz, z, pr.t, pr.a, pr.kall)
    assert np.max(np.abs(Fh - Fg)) <= 1e-4 * np.max(np.abs(Fg))


def test_rs_tucker_forces_converge_with_eps():
    """The adjoint forces of the RS-Tucker tensor (Tucker long part through the continuous basis
    functions, windows for the short part) tend to the forces of the untruncated Galerkin kernel
    as eps decreases: the error is of order eps down to 1e-8."""
    cfg = small_cfg()
    rng = np.random.default_rng(3)
    xyz = rng.uniform(-2.5, 2.5, (6, 3))
    z = rng.uniform(-1, 1, 6)
    pr = O.Problem(cfg, xyz, z)
    F = pr.forces_galerkin()
    errs = []
    for e in (1e-4, 1e-6, 1e-8):
        Ft, _ = pr.forces_rs_tucker(eps=e)
        errs.append(np.linalg.norm(Ft - F) / np.linalg.norm(F))
    assert errs[0] <= 3e-3 and errs[1] <= 1e-5 and errs[2] <= 1e-6, errs
    assert errs[2] < errs[1] < errs[0]


def test_direct_long_forces_equal_galerkin_up_to_window_cut():
    """Untruncated long-range pair forces plus the windows equal the Galerkin pair forces of the
    whole kernel except for the window cut-off (each cut term is below delta)."""
    cfg = small_cfg()
    rng = np.random.default_rng(3)
    xyz = rng.uniform(-2.5, 2.5, (6, 3))
    z = rng.uniform(-1, 1, 6)
    pr = O.Problem(cfg, xyz, z)
    F = pr.forces_galerkin()
    Fd = pr.forces_direct_long()
    assert np.linalg.norm(Fd - F) / np.linalg.norm(F) <= 1e-7


# ---------------------------------------------------------------- Def. 3.7, Lemma 3.8: Tucker-to-canonical
def _random_tucker(rng, n, ranks):
    Vs = [np.linalg.qr(rng.standard_normal((n, r)))[0] for r in ranks]
    # a graded core (decaying slices and singular values), like an RHOSVD core
    beta = rng.standard_normal(ranks) * np.exp(-0.7 * np.add.outer(np.add.outer(
        np.arange(ranks[0]), np.arange(ranks[1])), np.arange(ranks[2])))
    return beta, Vs


@pytest.mark.parametrize("eps", [0.0, 1e-6, 1e-3, 0.1])
def test_tucker_to_canonical_error_is_the_discarded_energy(eps):
    """Brute force on a 13^3 grid: ||T - C||_F^2 equals the discarded squared singular values,
    which stay within eps^2 ||T||_F^2, and discarding the smallest kept term would exceed it
    (the budget is used up); eps = 0 reproduces T exactly."""
    rng = np.random.default_rng(11)
    beta, Vs = _random_tucker(rng, 13, (5, 6, 4))
    xi, Us, kept, disc = O.tucker_to_canonical(beta, Vs, eps)
    T = np.einsum("abc,ia,jb,kc->ijk", beta, *Vs)          # full tensors, written out here
    C = sum(xi[k] * np.einsum("i,j,l->ijl", Us[0][:, k], Us[1][:, k], Us[2][:, k]) for k in range(len(xi)))
    C = np.asarray(C) if len(xi) else np.zeros_like(T)
    err2 = float(np.sum((T - C) ** 2))
    nT2 = float(np.sum(T * T))
    assert abs(err2 - disc) <= 1e-12 * nT2
    assert err2 <= eps * eps * nT2 * (1 + 1e-12) + 1e-28
    if eps == 0.0:
        assert np.abs(T - C).max() <= 1e-13 * np.abs(T).max()
        assert len(kept) == 5 * 4
    elif len(xi):
        assert disc + float(np.min(xi)) ** 2 > eps * eps * nT2


def test_tucker_to_canonical_known_rank():
    """A core that is a sum of three rank-1 terms in distinct mode-1 slices has RS-canonical
    rank 3 at any small eps, and its terms are recovered up to sign."""
    rng = np.random.default_rng(12)
    n = 9
    Vs = [np.linalg.qr(rng.standard_normal((n, r)))[0] for r in (4, 5, 5)]
    beta = np.zeros((4, 5, 5))
    lam = [3.0, -1.5, 0.25]
    for a, l in zip([0, 2, 3], lam):
        x, y = rng.standard_normal(5), rng.standard_normal(5)
        beta[a] += l * np.outer(x / np.linalg.norm(x), y / np.linalg.norm(y))
    xi, Us, kept, disc = O.tucker_to_canonical(beta, Vs, 1e-8)
    assert len(xi) == 3 and sorted(a for a, _ in kept) == [0, 2, 3]
    assert np.allclose(sorted(xi), sorted(abs(l) for l in lam))
    assert disc <= 1e-20


def test_canonical_points_match_full_tensor():
    """Lemma 3.8 (first term): the entry at i is the Hadamard product of the side-matrix rows
    times xi — against the full canonical tensor and against the Tucker tensor within the
    discarded energy."""
    rng = np.random.default_rng(13)
    beta, Vs = _random_tucker(rng, 11, (4, 4, 5))
    xi, Us, kept, disc = O.tucker_to_canonical(beta, Vs, 1e-4)
    C = O.canonical_full(xi, Us)
    idx = rng.integers(0, 11, (200, 3))
    v = O.canonical_points(xi, Us, idx)
    assert np.allclose(v, C[idx[:, 0], idx[:, 1], idx[:, 2]], rtol=0, atol=1e-14 * np.abs(C).max())
    T = O.tucker_points(beta, Vs, idx)
    assert np.abs(v - T).max() <= math.sqrt(disc) + 1e-14


# ---------------------------------------------------------------- Sec. 6 steps (III)-(V): ALS
@pytest.fixture(scope="module")
def small_problem():
    rng = np.random.default_rng(21)
    cfg = small_cfg()
    xyz, z = random_particles(rng, 6, 3.0, 1.0)
    pr = O.Problem(cfg, xyz, z)
    return pr, pr.Pl_grid()


def _unfold_projected(T, Vs, l):
    """Mode-l unfolding of T projected onto the bases of the two other modes, computed on the
    dense tensor (columns ordered by the lower other mode first)."""
    if l == 0:
        return np.einsum("ijk,jb,kc->ibc", T, Vs[1], Vs[2]).reshape(T.shape[0], -1)
    if l == 1:
        return np.einsum("ijk,ia,kc->jac", T, Vs[0], Vs[2]).reshape(T.shape[1], -1)
    return np.einsum("ijk,ia,jb->kab", T, Vs[0], Vs[1]).reshape(T.shape[2], -1)


def test_als_mode_matrix_is_the_projected_dense_unfolding(small_problem):
    """Step (IV): M_{U_l} is the partially projected image of the full tensor, reshaped.  Checked
    against the dense long-range tensor (pinned by brute force above), projected with random
    orthonormal bases that do not come from the oracle."""
    pr, Pl = small_problem
    Us, xi = O.side_matrices(pr.j, pr.z, pr.pk, pr.klong, pr.n)
    rng = np.random.default_rng(22)
    Vs = [np.linalg.qr(rng.standard_normal((pr.n, r)))[0] for r in (5, 7, 6)]
    for l in range(3):
        M = O.als_mode_matrix(Us, xi, Vs, l)
        D = _unfold_projected(Pl, Vs, l)
        assert M.shape == D.shape
        assert np.abs(M - D).max() <= 1e-12 * np.abs(D).max()


@pytest.mark.parametrize("fixed", [True, False])
def test_als_matches_dense_hooi(small_problem, fixed):
    """Steps (III)-(V) against textbook higher-order orthogonal iteration on the dense tensor.
    It starts from the same RHOSVD bases and updates the modes in order, each from the SVD of the
    projected unfolding (numpy on the dense tensor).  The bases (as projectors), ranks and core
    norm agree."""
    pr, Pl = small_problem
    eps = 1e-4
    Z0s, _, rk0, _, Us, xi = pr.tucker(eps=eps, cap=0)
    ranks = [max(2, r - 2) for r in rk0] if fixed else None
    Vs, beta, rk = O.c2t_als(Us, xi, Z0s, eps, 0, sweeps=2, ranks=ranks)
    D = [Z.copy() for Z in Z0s]
    rd = list(rk0)
    for _ in range(2):
        for l in range(3):
            W, s, _ = np.linalg.svd(_unfold_projected(Pl, D, l), full_matrices=False)
            if ranks is None:
                e2 = s ** 2
                tail = np.concatenate([np.cumsum(e2[::-1])[::-1], [0.0]])
                r = max(1, int(np.argmax(tail <= (eps * eps / 3.0) * e2.sum())))
            else:
                r = ranks[l]
            D[l] = W[:, :r]
            rd[l] = r
    assert rk == rd
    for V, W in zip(Vs, D):
        assert np.abs(V @ V.T - W @ W.T).max() <= 1e-9
    core = np.einsum("ijk,ia,jb,kc->abc", Pl, D[0], D[1], D[2])
    assert abs(np.linalg.norm(beta) - np.linalg.norm(core)) <= 1e-12 * np.linalg.norm(core)


def test_als_full_rank_is_exact(small_problem):
    """At full rank every projector is the identity on the column space: exact reconstruction."""
    pr, Pl = small_problem
    Z0s, _, _, _, Us, xi = pr.tucker(ranks=[pr.n] * 3)
    Vs, beta, rk = O.c2t_als(Us, xi, Z0s, 0.0, 0, sweeps=1, ranks=[pr.n] * 3)
    assert np.max(np.abs(O.tucker_full(beta, Vs) - Pl)) <= 1e-11 * np.max(np.abs(Pl))


def test_als_fixed_ranks_never_worse_and_monotone(c1_problem):
    """Each mode update of step (IV) maximises ||U x_1 P1 x_2 P2 x_3 P3|| over the projector of its
    mode with the others fixed, so at fixed ranks ||beta|| does not decrease from the RHOSVD start
    (Def. 6.1) or from one sweep to the next.  The Tucker error (full grid, with Pythagoras)
    therefore does not increase either."""
    pr, Pl = c1_problem
    Z0s, beta0, rk0, _, Us, xi = pr.tucker(eps=1e-5, cap=0)
    nrm = np.linalg.norm(Pl)
    e0 = np.linalg.norm(Pl - O.tucker_full(beta0, Z0s))
    b_prev = np.linalg.norm(beta0)
    for sweeps in (1, 2):
        Vs, beta, rk = O.c2t_als(Us, xi, Z0s, 1e-5, 0, sweeps=sweeps, ranks=rk0)
        assert rk == rk0
        b = np.linalg.norm(beta)
        assert b >= b_prev * (1 - 1e-14)
        b_prev = b
        err = np.linalg.norm(Pl - O.tucker_full(beta, Vs))
        assert err <= e0 * (1 + 1e-9)
        assert abs(nrm ** 2 - b * b - err ** 2) <= 1e-9 * nrm ** 2


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_als_eps_ranks_within_eps(c1_problem, eps):
    """The eps-truncation variant of the ALS (Sec. 6, remark after step (V)) keeps the Tucker error
    of the long part within eps on the full grid.  On this workload its ranks are at most the
    RHOSVD ranks in every mode and lower in total."""
    pr, Pl = c1_problem
    Z0s, _, rk0, _, Us, xi = pr.tucker(eps=eps, cap=0)
    Vs, beta, rk = O.c2t_als(Us, xi, Z0s, eps, 0, sweeps=1)
    err = np.linalg.norm(Pl - O.tucker_full(beta, Vs)) / np.linalg.norm(Pl)
    assert err <= eps
    assert all(a <= b for a, b in zip(rk, rk0)) and sum(rk) < sum(rk0)
    for V in Vs:
        assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)


# ---------------------------------------------------------------- discrete gradient (Sec. 4.3)
def test_fd_weights_closed_forms_and_polynomial_exactness():
    """The Taylor-condition weights reproduce the textbook centred formulas of orders 2 and 4, and
    every row of D_h (centred in the interior, one-sided at the ends) differentiates polynomials
    of degree <= order exactly."""
    h = 0.3
    w2 = O.fd_first_derivative_weights([-1, 0, 1], h)
    assert np.allclose(w2 * h, [-0.5, 0.0, 0.5], rtol=0, atol=1e-14)
    w4 = O.fd_first_derivative_weights([-2, -1, 0, 1, 2], h)
    assert np.allclose(w4 * h, [1 / 12, -2 / 3, 0.0, 2 / 3, -1 / 12], rtol=0, atol=1e-13)
    n, order = 23, 8
    D = O.fd_matrix(n, h, order)
    x = h * np.arange(n)
    xm, sc = x[n // 2], x[-1] / 2
    for q in range(order + 1):
        f = ((x - xm) / sc) ** q
        df = q * ((x - xm) / sc) ** max(q - 1, 0) / sc if q > 0 else np.zeros(n)
        assert np.abs(D @ f - df).max() <= 1e-8 * max(1.0, np.abs(df).max()), q
    # centred rows are antisymmetric about their point; each row sums to zero
    i = n // 2
    assert np.allclose(D[i, i - 4:i + 5], -D[i, i - 4:i + 5][::-1], rtol=0, atol=1e-12 / h)
    assert np.abs(D.sum(1)).max() <= 1e-11 / h


def test_fd_forces_converge_to_the_analytic_long_range_forces(c1_problem):
    """Forces from the discrete gradient of the untruncated long-range sum approach the forces
    from the analytic derivative of the Galerkin factors (rs_direct_long_forces) as the order
    of the difference formula rises."""
    pr = c1_problem[0]
    Fa = pr.forces_direct_long()
    errs = [np.linalg.norm(pr.forces_canonical_fd(order) - Fa) / np.linalg.norm(Fa) for order in (2, 4, 6, 8)]
    assert all(b < a / 8 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs


def test_fd_forces_converge_with_the_mesh_size():
    """Second-order centred differences: halving h divides the error of the discrete gradient of
    the long-range kernel by about four (same centres, same quadrature, grids n = 33, 65, 129)."""
    xyz = np.array([[0.5, -1.0, 1.5], [-1.5, 0.5, -0.5], [1.0, 1.0, -1.0]])
    z = np.array([0.8, -0.6, 0.4])
    errs = []
    for n in (33, 65, 129):
        pr = O.Problem(dict(b=4.0, n=n, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0,
                            delta_rel=1e-8), xyz, z)
        Fa = pr.forces_direct_long()
        errs.append(np.linalg.norm(pr.forces_canonical_fd(2) - Fa) / np.linalg.norm(Fa))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0, errs


def test_tucker_fd_forces_exact_at_full_rank_and_within_eps(c1_problem):
    """The discrete gradient applied to the Tucker form equals the discrete gradient of the
    canonical sum at full rank, and approaches it as eps falls (within 10 eps here: the
    difference operator weighs the discarded, more oscillatory directions by up to ~1/h)."""
    pr = c1_problem[0]
    Fc = pr.forces_canonical_fd(8)
    Ff, _ = pr.forces_rs_tucker_fd(ranks=[60, 60, 60])
    assert np.linalg.norm(Ff - Fc) <= 1e-12 * np.linalg.norm(Fc)
    for eps in (1e-4, 1e-6):
        Ft, _ = pr.forces_rs_tucker_fd(eps=eps)
        assert np.linalg.norm(Ft - Fc) <= 10 * eps * np.linalg.norm(Fc), eps


def test_fd_forces_momentum_and_self_term():
    """Centred differences of an even kernel are odd, so the forces of particles away from the
    ends of the grid add up to zero and a particle's own term has zero centred derivative; a
    one-sided row gives its own term a small, nonzero derivative."""
    rng = np.random.default_rng(41)
    xyz, z = random_particles(rng, 7, 2.5, 0.8)
    pr = O.Problem(small_cfg(), xyz, z)
    F = pr.forces_canonical_fd(8)
    assert np.abs(F.sum(0)).max() <= 1e-12 * np.abs(F).max()
    D = pr.fd_matrix(8)
    s = O.fd_self_gradient(pr.j, pr.pk, pr.klong, D)
    assert np.abs(s).max() <= 1e-14 * pr.PRl0 / pr.h
    jb = np.array([[0, pr.n // 2, pr.n // 2]])
    sb = O.fd_self_gradient(jb, pr.pk, pr.klong, D)
    tiny = 1e-14 * pr.PRl0 / pr.h
    assert abs(sb[0, 1]) <= tiny and abs(sb[0, 2]) <= tiny and abs(sb[0, 0]) > 100 * tiny, sb


# ---------------------------------------------------------------- RS interaction matrix (Sec. 4.1, 4.2)
@pytest.fixture(scope="module")
def matvec_problem():
    rng = np.random.default_rng(3)
    cfg = small_cfg(b=2.0, n=11, R=10, R_s=3, h_q=0.8, u0=-4.0, delta_rel=1e-6)
    xyz, z = random_particles(rng, 6, 1.8, 0.7)
    pr = O.Problem(cfg, xyz, z)
    A = O.rs_matrix_dense(pr.pk, pr.klong, pr.kshort, pr.gamma, pr.n)
    return pr, A


def test_rs_matrix_is_symmetric_translation_invariant_kronecker(matvec_problem):
    """A = A^T; an entry depends only on the difference of the two multi-indices (the d-level
    Toeplitz structure of Sec. 4.1, case (A)); the diagonal is P_R(0); the short part vanishes
    outside the window; on a 3-point grid the long part equals the brute-force sum of
    separable products."""
    pr, A = matvec_problem
    n = pr.n
    assert np.array_equal(A, A.T)
    idx = np.stack(np.unravel_index(np.arange(n ** 3), (n, n, n)), 1)
    rng = np.random.default_rng(5)
    for _ in range(200):
        a, b = rng.integers(0, n ** 3, 2)
        s = rng.integers(-2, 3, 3)
        ia, ib = idx[a] + s, idx[b] + s
        if np.all((ia >= 0) & (ia < n) & (ib >= 0) & (ib < n)):
            fa = np.ravel_multi_index(ia, (n, n, n))
            fb = np.ravel_multi_index(ib, (n, n, n))
            assert A[fa, fb] == A[a, b]
    assert np.allclose(np.diag(A), pr.PR0, rtol=1e-14, atol=0)
    # far apart (outside the window) only the long terms remain
    i0 = np.ravel_multi_index((0, 0, 0), (n, n, n))
    i1 = np.ravel_multi_index((n - 1, 0, 0), (n, n, n))
    c = n - 1
    assert abs(A[i0, i1] - sum(pr.pk[k, c - (n - 1)] * pr.pk[k, c] ** 2 for k in pr.klong)) <= 1e-15 * A[i0, i0]
    # 3-point grid: every entry from its definition, k by k
    m = 3
    t, a = O.sinc_quadrature(4, 0.9, -2.0)
    pk = O.reference_factors(t, a, 0.5, m)
    A3 = O.rs_matrix_dense(pk, np.arange(4), np.arange(0), 0, m)
    for p in range(m ** 3):
        for q in range(m ** 3):
            ip, iq = np.unravel_index(p, (m, m, m)), np.unravel_index(q, (m, m, m))
            ref = sum(np.prod([pk[k, ip[l] - iq[l] + m - 1] for l in range(3)]) for k in range(4))
            assert abs(A3[p, q] - ref) <= 1e-15 * abs(ref)


def test_rs_matvec_of_the_charges_is_the_rs_canonical_tensor(matvec_problem):
    """A applied to the charges embedded in the grid is the untruncated long-range canonical sum
    plus the windows of the cumulated canonical tensor (Eq. (3.5) and Defs. 3.4, 3.6, computed by
    their own functions): the matrix form of the RS tensor."""
    pr, A = matvec_problem
    C = O.charge_grid(pr.j, pr.z, pr.n)
    Y = (A @ C.ravel()).reshape(C.shape)
    ref = pr.Pl_grid() + pr.windows_grid()
    assert np.abs(Y - ref).max() <= 1e-14 * np.abs(ref).max()
    Y2 = O.rs_matvec_dense(pr.pk, pr.klong, pr.kshort, pr.gamma, pr.n, C, offdiag=True)
    assert np.abs(Y2 - (Y - pr.PR0 * C)).max() <= 1e-14 * np.abs(ref).max()


def test_energy_through_the_matrix(matvec_problem):
    """E_N = 1/2 <(A - diag A) z, z> (Eq. (4.6)) equals Eq. (4.7) on the RS tensor at the
    particles, the pair energy of the Galerkin kernel up to the window cut of the short terms,
    and the direct Coulomb energy within the quadrature error."""
    pr, _ = matvec_problem
    E = O.energy_matvec(pr.pk, pr.klong, pr.kshort, pr.gamma, pr.n, pr.j, pr.z)
    E47 = O.energy_from_potential(pr.Pl_points(pr.j) + pr.windows_points(pr.j), pr.z, pr.PR0)
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    assert abs(E - E47) <= 1e-13 * scale
    Ep = O.galerkin_pair_energy(pr.xyz_snapped, pr.z, pr.t, pr.a, pr.kall, pr.h)
    zz = float(np.sum(np.abs(np.outer(pr.z, pr.z))))
    assert abs(E - Ep) <= pr.delta * zz + 1e-13 * scale
    assert abs(E - pr.energy_direct_snapped()) <= 0.1 * scale
