"""GPU tests of the RS-canonical form (Def. 3.7, Lemma 3.8): the Tucker-to-canonical transform
of a solve's long part (slice SVD of the core, the smallest singular values discarded within
eps^2 ||beta||^2) against the oracle's transform of the same core and bases, its point values
against the oracle and against the RS-Tucker values of the same solve, and its edge cases.

Tolerances: the GPU SVD (one-sided Jacobi) and numpy's agree to FP64 rounding, so the ranks
are equal and the point values agree to 1e-10 of the largest value; against the Tucker
values of the same solve the difference is at most the discarded Frobenius norm
(max-abs <= Frobenius), sqrt(discarded) <= eps ||beta||_F.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402

pytestmark = pytest.mark.gpu


def _solve(cfg, p):
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    ctx = RSContext(config_from_workload(cfg, max_particles=max(1, len(p.Z))))
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"), energy=False,
              want_potential=False)
    torch.cuda.synchronize()
    return ctx


def _tucker64(ctx):
    """The solve's FP64 core and bases (what the transform reads)."""
    rk = ctx.report()["ranks"]
    n = ctx.n
    Z64 = ctx.debug_buffer("Z64", torch.float64)
    rmax = Z64.numel() // (3 * n)                 # the buffer is 3 x n x rmax
    Z64 = Z64[: 3 * n * rmax].view(3, n, rmax)
    b64 = ctx.debug_buffer("beta64", torch.float64)[: rmax ** 3].view(rmax, rmax, rmax)
    beta = b64[: rk[0], : rk[1], : rk[2]].cpu().numpy()
    Vs = [Z64[l, :, : rk[l]].cpu().numpy() for l in range(3)]
    return rk, beta, Vs


def _points(pr, rng, m=2000):
    return np.concatenate([pr.j, rng.integers(0, pr.n, (m, 3))])


@pytest.mark.parametrize("name,eps", [("c1_box64_n129", 1e-6), ("c1_box64_n129", 1e-3),
                                      ("c2_protein1000_n513", 4e-6)])
def test_canonical_matches_oracle_transform(name, eps):
    cfg = dict(load_config(name))
    cfg["rank_cap"] = 0
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _solve(cfg, p)
    rk, beta, Vs = _tucker64(ctx)
    xi, Us, kept, disc = O.tucker_to_canonical(beta, Vs, eps)
    R = ctx.canonical(eps)
    assert R == len(xi), (R, len(xi))
    rng = np.random.default_rng(5)
    idx = _points(pr, rng)
    it = torch.tensor(idx, device="cuda", dtype=torch.int32)
    got = ctx.canonical_eval_points(it).cpu().numpy()
    ref = O.canonical_points(xi, Us, idx) + O.windows_points(pr.j, pr.z, pr.pk, pr.kshort, pr.gamma, idx)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-10 * scale
    # the stored form itself (weights and side matrices) against the oracle's values
    gxi, gU = ctx.get_canonical()
    gxi = gxi.cpu().numpy()
    gU = [u.cpu().numpy() for u in gU]
    assert len(gxi) == R and all(u.shape == (pr.n, R) for u in gU)
    assert np.abs(O.canonical_points(gxi, gU, idx) - O.canonical_points(xi, Us, idx)).max() <= 1e-10 * scale
    # within the discarded energy of the Tucker values of the same solve (which the FP32 bulk
    # path evaluates from its FP32 T1, about 1e-7 relative)
    tuck = ctx.eval_points(it).cpu().numpy()
    rounding = 1e-12 if cfg["precision"] == "fp64" else 1e-6
    assert np.abs(got - tuck).max() <= np.sqrt(disc) * (1 + 1e-9) + rounding * scale
    ctx.close()


def test_canonical_rank_falls_with_eps_and_is_exact_at_zero():
    cfg = dict(load_config("c1_box64_n129"))
    cfg["rank_cap"] = 0
    p = make_particles(cfg)
    ctx = _solve(cfg, p)
    rk, beta, Vs = _tucker64(ctx)
    ranks = [ctx.canonical(e) for e in (0.0, 1e-8, 1e-6, 1e-4, 1e-2)]
    assert all(a >= b for a, b in zip(ranks, ranks[1:])), ranks
    # eps = 0 keeps every term of nonzero singular value: r1 min(r2, r3) of them (the Jacobi
    # SVD has r3 columns per slice, the r3 - r2 surplus ones of rounding size when r3 > r2)
    assert rk[0] * min(rk[1], rk[2]) <= ranks[0] <= rk[0] * rk[2]
    pr = O.Problem(cfg, p.xyz, p.Z)
    idx = _points(pr, np.random.default_rng(6), 500)
    it = torch.tensor(idx, device="cuda", dtype=torch.int32)
    ctx.canonical(0.0)
    got = ctx.canonical_eval_points(it).cpu().numpy()
    tuck = ctx.eval_points(it).cpu().numpy()
    assert np.abs(got - tuck).max() <= 1e-11 * np.abs(tuck).max()
    ctx.close()


def test_canonical_needs_its_solve():
    from paper_1606_09218_gb300 import RSError
    cfg = dict(load_config("c1_box64_n129"))
    cfg["rank_cap"] = 0
    p = make_particles(cfg)
    ctx = _solve(cfg, p)
    it = torch.zeros((4, 3), device="cuda", dtype=torch.int32)
    with pytest.raises(RSError):
        ctx.canonical_eval_points(it)
    ctx.canonical(1e-6)
    ctx.canonical_eval_points(it)
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"), energy=False,
              want_potential=False)
    with pytest.raises(RSError):                  # a new solve invalidates the form
        ctx.canonical_eval_points(it)
    with pytest.raises(RSError):
        ctx.canonical(-1.0)
    ctx.close()


def test_canonical_repeatable():
    """The transform is deterministic: the same rank and bit-identical values twice."""
    cfg = dict(load_config("c2_protein1000_n513"))
    p = make_particles(cfg)
    ctx = _solve(cfg, p)
    pr = O.Problem(cfg, p.xyz, p.Z)
    it = torch.tensor(_points(pr, np.random.default_rng(7), 300), device="cuda", dtype=torch.int32)
    r1 = ctx.canonical(4e-6)
    v1 = ctx.canonical_eval_points(it).clone()
    r2 = ctx.canonical(4e-6)
    v2 = ctx.canonical_eval_points(it)
    assert r1 == r2 and torch.equal(v1, v2)
    ctx.close()
