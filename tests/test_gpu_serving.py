"""GPU tests of the continuous-batching request loop (``rs_server_*``) on configuration-4
shaped requests (N up to 5000, n in {129, 257, 513}): each result is the same alone and in the
mix, admission respects the HBM budget and the slot limit, and served potentials and energies
match the oracle within the FP32 serving tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_serving_requests  # noqa: E402

pytestmark = pytest.mark.gpu

SERVE_TOL = 1e-4      # FP32 serving path, relative to the energy scale sum |z_j z_k| / r_jk


N_MAX = 5000          # the serving workload draws N log-uniform in [50, 5000]


def _requests(count, nmax, nmin=0, seed=4242):
    cfg = load_config("c4_serving256")
    reqs = [r for r in make_serving_requests(cfg, seed=seed, count=max(48, 4 * count)) if nmin <= r.n <= nmax]
    return cfg, reqs[:count]


def _cfg(cfg, n):
    from paper_1606_09218_gb300 import config_from_workload
    return config_from_workload(cfg, n=n, max_particles=N_MAX)


def _problem(cfg, r):
    c = dict(cfg)
    c.update(cfg["quad_by_n"][str(r.n)])
    c["n"] = r.n
    return O.Problem(c, r.particles.xyz, r.particles.Z)


def test_results_same_alone_and_in_mix():
    """Every request computes its potential (the tensor-core assembly runs concurrently for
    grids of different sizes) and its energy; the mix gives the results of the lone runs,
    bit for bit."""
    from paper_1606_09218_gb300 import RSServer
    cfg, reqs = _requests(12, 513)
    assert len(reqs) >= 8 and len({r.n for r in reqs}) >= 3
    srv = RSServer(hbm_budget=24 << 30, max_slots=6)
    alone = []
    pots_alone = []
    for r in reqs:
        pot = torch.empty((r.n,) * 3, dtype=torch.float32, device="cuda")
        res = srv.wait(srv.submit(_cfg(cfg, r.n), r.particles.xyz, r.particles.Z, potential=pot))
        assert res["status"] >= 0, res
        alone.append(res)
        pots_alone.append(pot)
    pots_mix = [torch.empty((r.n,) * 3, dtype=torch.float32, device="cuda") for r in reqs]
    tickets = [srv.submit(_cfg(cfg, r.n), r.particles.xyz, r.particles.Z, potential=pots_mix[i])
               for i, r in enumerate(reqs)]
    mix = [srv.wait(t) for t in tickets]
    info = srv.info()
    assert info["slots"] <= 6 and info["bytes_in_use"] <= (24 << 30)
    # more than one slot ran in the mix: the requests overlapped on the device
    assert len({m["slot"] for m in mix}) > 1
    # every sum of the path has a fixed order or is exact: the mix reproduces the lone runs bit
    # for bit
    for r, a, m in zip(reqs, alone, mix):
        assert m["status"] == a["status"] and m["ranks"] == a["ranks"], (a, m)
        assert m["energy"] == a["energy"], (a, m)
    for pa, pm in zip(pots_alone, pots_mix):
        assert torch.equal(pa, pm)
    srv.close()


def test_contexts_of_different_sizes_interleave():
    """A context keeps working after a context of another grid size has run: the kernels'
    launch limits are per process, not per context."""
    from paper_1606_09218_gb300 import RSContext
    cfg, reqs = _requests(48, 513)
    big = next(r for r in reqs if r.n == 513)
    small = next(r for r in reqs if r.n == 129)
    a = RSContext(_cfg(cfg, 513))
    pa = a.new_potential()
    a.solve(big.particles.xyz, big.particles.Z, potential=pa, energy=True)
    Ea = a.energy()
    first = pa.clone()
    b = RSContext(_cfg(cfg, 129))
    pb = b.new_potential()
    b.solve(small.particles.xyz, small.particles.Z, potential=pb, energy=True)
    b.energy()
    a.solve(big.particles.xyz, big.particles.Z, potential=pa, energy=True)
    assert abs(a.energy() - Ea) <= 1e-12 * abs(Ea) + 1e-12
    assert float((pa - first).abs().max()) <= 1e-6 * float(first.abs().max())
    assert a.report()["status"] >= 0
    a.close()
    b.close()


def test_admission_by_footprint_serialises_within_budget():
    """A budget that holds one n = 257 workspace at a time still serves every request."""
    import ctypes as C
    from paper_1606_09218_gb300 import RSServer, _lib
    cfg, reqs = _requests(6, 257)
    lib = _lib.load()
    need = max(lib.rs_workspace_bytes(C.byref(_cfg(cfg, r.n))) for r in reqs)
    srv = RSServer(hbm_budget=int(need * 1.2), max_slots=4)
    tickets = [srv.submit(_cfg(cfg, r.n), r.particles.xyz, r.particles.Z) for r in reqs]
    res = [srv.wait(t) for t in tickets]
    assert all(r["status"] >= 0 for r in res)
    assert srv.info()["bytes_in_use"] <= int(need * 1.2)
    srv.close()


def test_served_potentials_and_energies_match_oracle():
    """One request per grid size (n = 129, 257, 513), the largest N of each size among the first
    48 requests of the workload's generator (N up to 5000): the served potential against the
    oracle's full-rank canonical sum P_0 at every charged site and 1500 random grid points, and the
    served energy against the oracle's energy of P_0 (Eq. (4.7)), both within the FP32 serving
    tolerance 1e-4 (relative Frobenius over the sample; energy relative to sum |z_j z_k| / r_jk).
    The error budget is eps ||P_l|| (Tucker) + the window cut-off + FP32 rounding, about 1e-6."""
    from paper_1606_09218_gb300 import RSServer
    cfg, reqs = _requests(48, 513)
    chosen = []
    for n in (129, 257, 513):
        cand = [r for r in reqs if r.n == n]
        assert cand, n
        chosen.append(max(cand, key=lambda r: len(r.particles.Z)))
    assert max(len(r.particles.Z) for r in chosen) > 2000
    srv = RSServer(hbm_budget=16 << 30, max_slots=3)
    pots = [torch.empty((r.n,) * 3, dtype=torch.float32, device="cuda") for r in chosen]
    tickets = [srv.submit(_cfg(cfg, r.n), r.particles.xyz, r.particles.Z, potential=p) for r, p in zip(chosen, pots)]
    res = [srv.wait(t) for t in tickets]
    srv.close()
    rng = np.random.default_rng(99)
    for r, p, x in zip(chosen, pots, res):
        assert x["status"] >= 0, x
        pr = _problem(cfg, r)
        idx = np.concatenate([pr.j[pr.z != 0], rng.integers(0, r.n, (1500, 3))])
        it = torch.tensor(idx, device="cuda", dtype=torch.long)
        g = p[it[:, 0], it[:, 1], it[:, 2]].double().cpu().numpy()
        ref = pr.P0_points(idx)
        err = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        assert err < SERVE_TOL, (r.n, len(r.particles.Z), err)
        scale = O.energy_scale(pr.xyz_snapped, pr.z)
        E0 = O.energy_from_potential(pr.P0_points(pr.j), pr.z, pr.PR0)
        assert abs(x["energy"] - E0) <= SERVE_TOL * scale, (r.n, x["energy"], E0, scale)
