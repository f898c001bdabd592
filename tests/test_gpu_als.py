"""GPU parity of the ALS refinement of the canonical-to-Tucker transform (Sec. 6, steps
(III)-(V)) through the C ABI (rs_tucker_als), against the oracle's ALS (c2t_als) on the same
seeded inputs.

The GPU starts from its own RHOSVD ranks; the oracle starts from the RHOSVD at those ranks and,
for the comparison of tensors, takes the GPU's refined ranks (its own eps ranks must agree within
one per mode: a singular value at the cut may fall on either side in the two eigensolvers).
Tolerances as in the parity tests of the solve: both refined long parts lie within eps of the
untruncated one, so they agree within 2 eps ||P_l|| (relative to the grid) plus rounding (1e-9
FP64, 1e-6 FP32 bulk); energies within 1e-8 / 1e-6 of sum_{j<k} |z_j z_k| / r_jk.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(cfg, N):
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    return RSContext(config_from_workload(cfg, max_particles=max(1, N)))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check_against_oracle(cfg, pr, ctx, r0, rounding, sweeps=1):
    """The GPU's refined potential and energy against the oracle's ALS from the same start.
    After one sweep both took the same rank in every mode update; after more sweeps the oracle
    keeps the GPU's final ranks throughout, so only the potentials (both within eps of P_l) are
    compared."""
    rep = ctx.report()
    r1 = rep["ranks"]
    Z0s, _, _, _, Us, xi = pr.tucker(ranks=r0)
    _, _, rk_or = O.c2t_als(Us, xi, Z0s, cfg["eps"], cfg.get("rank_cap", 0), sweeps=sweeps)
    assert all(abs(a - b) <= 1 for a, b in zip(r1, rk_or)), (r1, rk_or)
    Vs, beta, _ = O.c2t_als(Us, xi, Z0s, cfg["eps"], 0, sweeps=sweeps, ranks=r1)
    W = pr.windows_grid()
    ref = O.tucker_full(beta, Vs) + W
    Pl = pr.Pl_grid()
    P = ctx.potential.double().cpu().numpy()
    tol = 2 * cfg["eps"] * np.linalg.norm(Pl) / np.linalg.norm(ref) + rounding
    assert _rel(P, ref) < tol
    # the refined long part stays within eps of the untruncated one
    assert np.linalg.norm((P - W) - Pl) <= cfg["eps"] * np.linalg.norm(Pl) + rounding * np.linalg.norm(ref)
    if sweeps == 1:
        A = O.tucker_points(beta, Vs, pr.j) + pr.windows_points(pr.j)
        Eref = O.energy_from_potential(A, pr.z, pr.PR0)
        scale = O.energy_scale(pr.xyz_snapped, pr.z)
        assert abs(ctx.energy() - Eref) <= (1e-8 if rounding < 1e-7 else 1e-6) * scale
    return r1


def test_c1_als_matches_oracle_and_lowers_ranks():
    """Configuration 1 without the rank cap (FP64): one sweep lowers the eps ranks and stays
    within eps; a second call continues from the refined form."""
    cfg = dict(load_config("c1_box64_n129"))
    cfg["rank_cap"] = 0
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"))
    r0 = ctx.report()["ranks"]
    ctx.tucker_als(1)
    r1 = _check_against_oracle(cfg, pr, ctx, r0, 1e-9)
    assert sum(r1) < sum(r0), (r0, r1)
    # Tucker bases stay orthonormal
    ranks, Vs, _ = ctx.tucker()
    assert list(ranks) == list(r1)
    for V in Vs:
        V = V.cpu().numpy()
        assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-12
    # second sweep through a second call
    ctx.tucker_als(1)
    _check_against_oracle(cfg, pr, ctx, r0, 1e-9, sweeps=2)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_small_random_problems_als(prec):
    """Ragged grids (n = 37, 45), overlapping windows, a zero charge, both precisions."""
    rng = np.random.default_rng(31)
    rnd = 1e-9 if prec == "fp64" else 1e-6
    for n, N in ((37, 7), (45, 19)):
        cfg = dict(b=4.0, n=n, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0,
                   delta_rel=1e-8, precision=prec, snap=True)
        xyz = rng.uniform(-4.0, 4.0, (N, 3))
        xyz[0] = [-4.0, 4.0, 0.0]
        Z = rng.uniform(-1, 1, N)
        Z[1] = 0.0
        pr = O.Problem(cfg, xyz, Z)
        ctx = _ctx(cfg, N)
        ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"))
        r0 = ctx.report()["ranks"]
        ctx.tucker_als(1)
        _check_against_oracle(cfg, pr, ctx, r0, rnd)
        ctx.close()


def test_als_over_several_k_chunks():
    """400 charges on the 129^3 grid with rank bound 128: the mode matrices are summed over two
    K chunks (the second one ragged), FP64."""
    cfg = dict(load_config("c1_box64_n129"))
    cfg["rank_cap"] = 0
    cfg["max_rank"] = 128
    cfg["particles"] = dict(cfg["particles"], N=400)
    p = make_particles(cfg, seed=77)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ncoord = [len(np.unique(pr.j[:, l])) for l in range(3)]
    assert min(ncoord) * (cfg["R"] - cfg["R_s"]) > (1 << 24) // (128 * 128)
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"))
    r0 = ctx.report()["ranks"]
    ctx.tucker_als(1)
    _check_against_oracle(cfg, pr, ctx, r0, 1e-9)
    ctx.close()


def test_als_reproducible_and_eval_points():
    """Two contexts, same input: bit-identical refined potentials; point values of the refined
    tensor equal its grid values; the RS-canonical form follows the refined core."""
    cfg = dict(b=4.0, n=45, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0,
               delta_rel=1e-8, precision="fp64", snap=True)
    rng = np.random.default_rng(32)
    xyz = rng.uniform(-3.5, 3.5, (12, 3))
    Z = rng.uniform(-1, 1, 12)
    outs = []
    for _ in range(2):
        ctx = _ctx(cfg, 12)
        ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"))
        ctx.tucker_als(2)
        outs.append((ctx.potential.clone(), ctx.energy(), ctx.report()["ranks"]))
        idx = rng.integers(0, 45, (300, 3))
        v = ctx.eval_points(torch.tensor(idx, dtype=torch.int32)).cpu().numpy()
        P = ctx.potential.cpu().numpy()
        assert np.abs(v - P[idx[:, 0], idx[:, 1], idx[:, 2]]).max() <= 1e-10 * np.abs(P).max()
        R = ctx.canonical(0.0)
        vc = ctx.canonical_eval_points(torch.tensor(idx, dtype=torch.int32)).cpu().numpy()
        assert R > 0 and np.abs(vc - v).max() <= 1e-10 * np.abs(P).max()
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]


def test_als_errors_and_no_charge():
    from paper_1606_09218_gb300 import RSError
    from paper_1606_09218_gb300._lib import RS_ERR_INVALID_ARG, RS_ERR_NOT_READY
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp64", snap=True)
    ctx = _ctx(cfg, 2)
    with pytest.raises(RSError) as e:
        ctx.tucker_als(1)
    assert e.value.status == RS_ERR_NOT_READY
    xyz = torch.tensor([[0.5, 0.5, 0.5], [-1.0, 2.0, 0.0]], dtype=torch.float64, device="cuda")
    ctx.solve(xyz, torch.tensor([0.7, -0.4], dtype=torch.float64, device="cuda"), energy=False)
    for bad in (0, 9):
        with pytest.raises(RSError) as e:
            ctx.tucker_als(bad)
        assert e.value.status == RS_ERR_INVALID_ARG
    with pytest.raises(RSError) as e:          # no solve energy to refine
        ctx.tucker_als(1, energy=True)
    assert e.value.status == RS_ERR_NOT_READY
    ctx.tucker_als(1, energy=False)
    # all charges zero: nothing to refine, the potential stays zero
    ctx.solve(xyz, torch.zeros(2, dtype=torch.float64, device="cuda"))
    ctx.tucker_als(1)
    assert float(ctx.potential.abs().max()) == 0.0 and ctx.energy() == 0.0
    ctx.close()
