"""Run-to-run reproducibility: repeated solves of the same input give bit-identical potentials,
energies and forces.  Every floating-point sum of the path has a fixed order or is exact:
the column weights and the Tucker core add 64-bit fixed-point integers atomically, the FP64
products split K through ordered partial tiles, and the other reductions have a fixed tree.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import load_config, make_particles, make_serving_requests  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(cfg, N, **kw):
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    return RSContext(config_from_workload(cfg, max_particles=N, **kw))


@pytest.mark.parametrize("name", ["c1_box64_n129", "c2_protein1000_n513"])
def test_repeated_solves_bit_identical(name):
    cfg = load_config(name)
    p = make_particles(cfg)
    ctx = _ctx(cfg, len(p.Z))
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    ref = None
    for _ in range(3):
        pot = ctx.new_potential()
        ctx.solve(xyz, Z, potential=pot, energy=True, forces=True)
        res = (pot, ctx.energy(), ctx.forces(), ctx.report()["ranks"])
        torch.cuda.synchronize()
        if ref is None:
            ref = res
            continue
        assert torch.equal(res[0], ref[0])
        assert res[1] == ref[1]
        assert torch.equal(res[2], ref[2])
        assert res[3] == ref[3]
    ctx.close()


def test_repeated_solves_bit_identical_tensor_core_core():
    """The 1025^3 lattice path (core contraction on the tensor cores) on a smaller lattice with
    the same tolerance: the fixed-point core sums make it reproducible as well."""
    cfg = dict(load_config("c3_nacl28_n1025"))
    cfg["n"] = 257
    cfg["particles"] = dict(cfg["particles"], side=10)
    p = make_particles(cfg)
    ctx = _ctx(cfg, len(p.Z))
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    pots, Es = [], []
    for _ in range(3):
        pot = ctx.new_potential()
        ctx.solve(xyz, Z, potential=pot, energy=True)
        Es.append(ctx.energy())
        pots.append(pot)
    torch.cuda.synchronize()
    assert Es[0] == Es[1] == Es[2]
    assert torch.equal(pots[0], pots[1]) and torch.equal(pots[0], pots[2])
    ctx.close()


def test_serving_shaped_requests_reproducible():
    """Small serving-shaped problems, where coordinates are shared by several particles (the
    case whose weight sums once depended on the order of the atomic additions)."""
    cfg = load_config("c4_serving256")
    reqs = [r for r in make_serving_requests(cfg, seed=4242, count=48) if r.n <= 257][:6]
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    for r in reqs:
        ctx = RSContext(config_from_workload(cfg, n=r.n, max_particles=len(r.particles.Z)))
        Es = []
        for _ in range(4):
            ctx.solve(r.particles.xyz, r.particles.Z, energy=True, want_potential=False)
            Es.append(ctx.energy())
        assert len(set(Es)) == 1, Es
        ctx.close()
