"""The seeded synthetic inputs follow their stated recipe (CPU).

Checked for every workload: counts, regions, minimum separations, charge sets and
distributions, lattice structure, serving arrivals and sizes, and reproducibility.  The
batched random sequential addition of the generator is compared with a one-candidate-at-a-time
version written here from the definition.  The two must give the same points and leave the
random stream at the same position.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from workloads import generate as Gen
from workloads import load_config, make_particles, make_serving_requests


def _min_dist(x):
    if len(x) < 2:
        return np.inf
    d, _ = cKDTree(x).query(x, k=2)
    return float(d[:, 1].min())


def _rsa_one_at_a_time(rng, n_pts, half, inside, sep):
    """Draw one candidate (three uniforms in [-half, half]) at a time; keep it if it lies in
    the region and at distance >= sep from every point kept before it."""
    pts = np.empty((0, 3))
    while len(pts) < n_pts:
        x = rng.uniform(-half, half, 3)
        if not inside(x):
            continue
        if len(pts):
            d = pts - x
            if np.min(np.einsum("ij,ij->i", d, d)) < sep * sep:
                continue
        pts = np.vstack([pts, x])
    return pts


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_c1_uniform_box():
    cfg = load_config("c1_box64_n129")
    p = make_particles(cfg)
    assert p.xyz.shape == (64, 3) and p.Z.shape == (64,)
    assert np.abs(p.xyz).max() <= 8.0 and _min_dist(p.xyz) >= 1.0
    assert np.abs(p.Z).max() <= 1.0 and len(np.unique(p.Z)) == 64


def test_c2_protein_ball_and_charge_distribution():
    cfg = load_config("c2_protein1000_n513")
    p = make_particles(cfg)
    assert p.xyz.shape == (1000, 3)
    assert np.linalg.norm(p.xyz, axis=1).max() <= 15.0 and _min_dist(p.xyz) >= 1.2
    vals = np.asarray(cfg["particles"]["charge_values"])
    probs = np.asarray(cfg["particles"]["charge_probs"])
    assert set(np.unique(p.Z)) <= set(vals)
    counts = np.array([(p.Z == v).sum() for v in vals])
    sd = np.sqrt(1000 * probs * (1 - probs))
    assert np.all(np.abs(counts - 1000 * probs) <= 5 * sd), counts


def test_c3_rock_salt_lattice_with_vacancies():
    cfg = load_config("c3_nacl28_n1025")
    p = make_particles(cfg)
    m = 28
    assert len(p.Z) == m ** 3 - int(round(0.1 * m ** 3)) == 19757
    idx = p.xyz + 13.5                                    # spacing 1.0, centred lattice
    assert np.allclose(idx, np.round(idx), atol=0) and idx.min() >= 0 and idx.max() <= m - 1
    ii = np.round(idx).astype(int)
    assert len(np.unique(ii[:, 0] * m * m + ii[:, 1] * m + ii[:, 2])) == len(ii)
    assert np.array_equal(p.Z, np.where(ii.sum(1) % 2 == 0, 1.0, -1.0))
    # nearest neighbours (distance 1) carry opposite charges
    pairs = cKDTree(p.xyz).query_pairs(1.0 + 1e-9, output_type="ndarray")
    assert len(pairs) > 0 and np.all(p.Z[pairs[:, 0]] * p.Z[pairs[:, 1]] == -1.0)


def test_c5_neutral_ball():
    cfg = load_config("c5_forces4096_n513")
    p = make_particles(cfg)
    assert p.xyz.shape == (4096, 3)
    assert np.linalg.norm(p.xyz, axis=1).max() <= 12.0 and _min_dist(p.xyz) >= 1.0
    assert set(np.unique(p.Z)) == {-1.0, 1.0} and p.Z.sum() == 0.0


def test_c4_serving_requests():
    cfg = load_config("c4_serving256")
    s = cfg["serving"]
    reqs = make_serving_requests(cfg)
    assert len(reqs) == 256
    t = np.array([r.arrival_s for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
    assert abs(np.diff(t).mean() - 2e-3) <= 0.25 * 2e-3        # Poisson, mean gap 2 ms
    Ns = np.array([len(r.particles.Z) for r in reqs])
    assert Ns.min() >= s["N_min"] and Ns.max() <= s["N_max"]
    # log-uniform: about half the requests below the geometric mean of the range
    assert abs(np.mean(Ns < np.sqrt(s["N_min"] * s["N_max"])) - 0.5) <= 0.15
    assert set(r.n for r in reqs) <= set(s["n_choices"]) and len(set(r.n for r in reqs)) == 3
    vol = (2 * s["half"]) ** 3
    for r in reqs:
        x = r.particles.xyz
        sep = min(s["min_sep"], 0.8 * (vol / len(x)) ** (1.0 / 3.0))
        assert np.abs(x).max() <= s["half"] and _min_dist(x) >= sep * (1 - 1e-12)
        assert np.abs(r.particles.Z).max() <= 1.0


def test_inputs_are_reproducible():
    for name in ("c1_box64_n129", "c2_protein1000_n513", "c3_nacl28_n1025"):
        cfg = load_config(name)
        a, b = make_particles(cfg), make_particles(cfg)
        assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.Z, b.Z)
    cfg = load_config("c4_serving256")
    r1 = make_serving_requests(cfg, count=8)
    r2 = make_serving_requests(cfg, count=8)
    assert all(np.array_equal(a.particles.xyz, b.particles.xyz) and a.n == b.n for a, b in zip(r1, r2))


@pytest.mark.parametrize("name", ["c1_box64_n129", "c2_protein1000_n513", "c5_forces4096_n513"])
def test_batched_rsa_equals_one_candidate_at_a_time(name):
    cfg = load_config(name)
    p = cfg["particles"]
    seed = Gen.seed_for(cfg["index"])
    N = int(p["N"])
    if p["kind"] == "uniform_box":
        half, inside = float(p["half"]), (lambda x: True)
    else:
        R = float(p["radius"])
        half, inside = R, (lambda x, R=R: float(x @ x) <= R * R)
    rng_ref = _rng(seed)
    ref = _rsa_one_at_a_time(rng_ref, N, half, inside, float(p["min_sep"]))
    rng = _rng(seed)
    attempts = Gen._box_attempts(half) if p["kind"] == "uniform_box" else Gen._ball_attempts(half)
    got = Gen._rsa(rng, N, attempts, float(p["min_sep"]))
    assert np.array_equal(got, ref)
    # the stream is left where the one-at-a-time draws left it
    assert rng.uniform() == rng_ref.uniform()
    assert np.array_equal(make_particles(cfg).xyz, ref)
