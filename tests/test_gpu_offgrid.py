"""GPU tests of the energy and forces at centres off the grid (rs_pair_energy_forces): the RS
kernel of the context in pair form against the oracle's Galerkin pair energy and forces, its
finite differences (h = 1e-4, far below the grid spacing), the RS grid path at snapped centres,
and the direct Coulomb forces of the forces workload (N = 4096) within the quadrature error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(cfg, N):
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    return RSContext(config_from_workload(cfg, max_particles=N))


def _cuda(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def test_pair_energy_forces_match_oracle():
    rng = np.random.default_rng(41)
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp32_split", snap=False)
    N = 40
    xyz = rng.uniform(-3.0, 3.0, (N, 3))
    Z = rng.uniform(-1, 1, N)
    Z[7] = 0.0
    ctx = _ctx(dict(cfg, snap=True), N)
    E, F = ctx.pair_energy_forces(_cuda(xyz), _cuda(Z))
    F = F.cpu().numpy()
    h = 2 * cfg["b"] / (cfg["n"] - 1)
    t, a = O.sinc_quadrature(cfg["R"], cfg["h_q"], cfg["u0"])
    ks = np.arange(cfg["R"])
    Eo = O.galerkin_pair_energy(xyz, Z, t, a, ks, h)
    Fo = O.galerkin_pair_forces(xyz, Z, t, a, ks, h)
    scale = O.energy_scale(xyz, Z)
    assert abs(E - Eo) <= 1e-6 * scale, (E, Eo)
    assert np.abs(F - Fo).max() <= 2e-6 * np.abs(Fo).max()
    assert np.all(F[7] == 0.0)
    ctx.close()


def test_pair_energy_continues_the_grid_path():
    """At snapped centres the pair form of the full Galerkin kernel and the RS-Tucker energy of a
    solve (long part at eps, windows cut at delta) agree within O(eps)."""
    rng = np.random.default_rng(43)
    cfg = dict(b=4.0, n=45, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp64", snap=True)
    N = 16
    xyz = rng.uniform(-3.2, 3.2, (N, 3))
    Z = rng.uniform(-1, 1, N)
    pr = O.Problem(cfg, xyz, Z)
    ctx = _ctx(cfg, N)
    ctx.solve(_cuda(pr.xyz_snapped), _cuda(Z), energy=True, want_potential=False)
    E_rs = ctx.energy()
    E_pair, _ = ctx.pair_energy_forces(_cuda(pr.xyz_snapped), _cuda(Z), forces=False)
    scale = O.energy_scale(pr.xyz_snapped, Z)
    assert abs(E_rs - E_pair) <= 20 * cfg["eps"] * scale, (E_rs, E_pair)
    ctx.close()


def test_c5_forces_full_size_fd_coulomb_momentum():
    """Forces workload at full size (N = 4096, neutral, unsnapped): total force zero, central
    finite differences (h = 1e-4) of the oracle's FP64 kernel for sampled particles, and the
    direct Coulomb forces within the error of the sinc quadrature and the cell averages."""
    cfg = load_config("c5_forces4096_n513")
    p = make_particles(cfg)
    N = len(p.Z)
    ctx = _ctx(dict(cfg, snap=True), N)
    E, F = ctx.pair_energy_forces(_cuda(p.xyz), _cuda(p.Z))
    F = F.cpu().numpy()
    assert np.isfinite(E) and np.all(np.isfinite(F))
    assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum()
    h = 2 * cfg["b"] / (cfg["n"] - 1)
    t, a = O.sinc_quadrature(cfg["R"], cfg["h_q"], cfg["u0"])
    ks = np.arange(cfg["R"])

    def e_j(j, x):
        y = x[None, :] - p.xyz
        f = [O.galerkin_factors_at(t, a, h, y[:, l]) for l in range(3)]
        K = (f[0] * f[1] * f[2]).sum(0)
        K[j] = 0.0
        return p.Z[j] * float(K @ p.Z)

    fd_h = 1e-4
    rng = np.random.default_rng(5)
    for j in rng.choice(N, 6, replace=False):
        for l in range(3):
            e = np.zeros(3)
            e[l] = fd_h
            fd = -(e_j(j, p.xyz[j] + e) - e_j(j, p.xyz[j] - e)) / (2 * fd_h)
            assert abs(F[j, l] - fd) <= 1e-5 * max(1.0, abs(fd)), (j, l, F[j, l], fd)
    Fc = O.forces_direct(p.xyz, p.Z)
    rel = np.linalg.norm(F - Fc) / np.linalg.norm(Fc)
    assert rel < 2e-2, rel
    Ec = O.energy_direct(p.xyz, p.Z)
    assert abs(E - Ec) <= 1e-2 * O.energy_scale(p.xyz, p.Z)
    ctx.close()
