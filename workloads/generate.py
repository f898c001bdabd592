"""Seeded generators for the five synthetic workloads.

Every generator uses numpy's PCG64 with ``seed = 160609218 + index`` (or a caller
seed) and returns float64 host arrays.  The shapes follow the particle systems the
paper evaluates (Sec. 3.1 protein-type clusters with a minimal inter-atomic
distance, Def. "well-separable point distribution"; the random-charge lattices of
Sec. 4.2, Table "EN_NU_LatRand"):

* ``uniform_box``: N points uniform in [-L, L]^3, random sequential addition with a
  minimum pair separation, charges uniform in [-1, 1];
* ``protein_ball``: N points uniform in a ball, minimum separation, charges drawn
  from a small discrete set;
* ``nacl_lattice``: a cubic lattice with alternating charges and random vacancies;
* ``neutral_ball``: N points in a ball, charges +1/-1 in equal numbers.

The module never touches the method (no quadrature, factors or sums).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

BASE_SEED = 160609218
_CFG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")

#: workload name -> parameter file
WORKLOADS = {
    "c1_box64_n129": "c1_box64_n129.json",
    "c2_protein1000_n513": "c2_protein1000_n513.json",
    "c3_nacl28_n1025": "c3_nacl28_n1025.json",
    "c4_serving256": "c4_serving256.json",
    "c5_forces4096_n513": "c5_forces4096_n513.json",
}


def seed_for(index: int) -> int:
    return BASE_SEED + int(index)


def load_config(name: str) -> dict:
    """Return the parameter dictionary of a workload (method and generator keys)."""
    fn = WORKLOADS.get(name, name)
    path = fn if os.path.isabs(fn) else os.path.join(_CFG_DIR, fn)
    with open(path) as f:
        return json.load(f)


def _rsa(rng: np.random.Generator, n_pts: int, attempts, sep: float, max_tries: int = 10_000_000):
    """Random sequential addition: draw candidates one after another and keep those at
    distance >= sep from every point accepted before them.

    ``attempts(rng, B)`` draws B raw attempts (B x 3, three uniform numbers each, in the same
    stream order as B single draws) and returns them with a mask of the attempts that are
    candidates (inside the region).  Attempts are drawn in batches and checked against the
    accepted points with a k-d tree, then in order against the points accepted earlier in the
    same batch; the generator is rewound to the attempts actually used, so the result and the
    stream position equal those of drawing one attempt at a time."""
    from scipy.spatial import cKDTree
    pts = np.zeros((n_pts, 3))
    count = 0
    tries = 0
    sep2 = sep * sep
    tree = None
    while count < n_pts:
        B = max(256, 4 * (n_pts - count))
        state = rng.bit_generator.state
        raw, valid = attempts(rng, B)
        far = np.ones(B, dtype=bool)
        if count > 0:
            _, idx = tree.query(raw, k=1)
            d = pts[idx] - raw
            far = np.einsum("ij,ij->i", d, d) >= sep2
        cand = np.flatnonzero(valid & far)
        # conflicts among this batch's candidates: earlier[i] lists the earlier candidates
        # closer than sep to candidate i
        earlier: dict[int, list[int]] = {}
        if len(cand) > 1:
            for a, b in cKDTree(raw[cand]).query_pairs(sep):
                i, j = cand[a], cand[b]
                if i > j:
                    i, j = j, i
                d = raw[i] - raw[j]
                if d @ d < sep2:
                    earlier.setdefault(int(j), []).append(int(i))
        accepted = set()
        new = []
        used = B
        for i in cand:
            i = int(i)
            if tries + i + 1 > max_tries:
                raise RuntimeError("random sequential addition did not reach the requested count")
            if any(j in accepted for j in earlier.get(i, ())):
                continue
            accepted.add(i)
            new.append(i)
            if count + len(new) == n_pts:
                used = i + 1
                break
        tries += used
        if tries > max_tries and count + len(new) < n_pts:
            raise RuntimeError("random sequential addition did not reach the requested count")
        pts[count:count + len(new)] = raw[new]
        count += len(new)
        if used < B:                       # rewind to the attempts actually used
            rng.bit_generator.state = state
            attempts(rng, used)
        tree = cKDTree(pts[:count])
    return pts


def _uniform_box(rng, half):
    return rng.uniform(-half, half, 3)


def _box_attempts(half):
    def f(rng, B):
        x = rng.uniform(-half, half, (B, 3))
        return x, np.ones(B, dtype=bool)
    return f


def _ball_attempts(radius):
    def f(rng, B):
        x = rng.uniform(-radius, radius, (B, 3))
        return x, np.einsum("ij,ij->i", x, x) <= radius * radius
    return f


def _uniform_ball(radius):
    def f(rng):
        while True:
            x = rng.uniform(-radius, radius, 3)
            if x @ x <= radius * radius:
                return x
    return f


@dataclass
class Particles:
    xyz: np.ndarray   # (N, 3) float64
    Z: np.ndarray     # (N,) float64


def make_particles(cfg: dict, seed: int | None = None) -> Particles:
    """Generate the particle set described by ``cfg['particles']``."""
    p = cfg["particles"]
    kind = p["kind"]
    rng = np.random.Generator(np.random.PCG64(seed_for(cfg["index"]) if seed is None else seed))
    if kind == "uniform_box":
        N = int(p["N"])
        # a minimum separation above what random sequential addition can reach (its jamming
        # packing fraction is about 0.38) is lowered to 0.8 (V/N)^{1/3}, packing fraction 0.27;
        # this only changes the largest serving requests (N above ~2000 in [-8, 8]^3)
        vol = (2.0 * float(p["half"])) ** 3
        sep = min(float(p["min_sep"]), 0.8 * (vol / max(N, 1)) ** (1.0 / 3.0))
        xyz = _rsa(rng, N, _box_attempts(p["half"]), sep)
        Z = rng.uniform(-1.0, 1.0, N)
    elif kind == "protein_ball":
        N = int(p["N"])
        xyz = _rsa(rng, N, _ball_attempts(p["radius"]), p["min_sep"])
        Z = rng.choice(np.asarray(p["charge_values"], float), size=N, p=np.asarray(p["charge_probs"], float))
    elif kind == "nacl_lattice":
        m = int(p["side"])
        a = float(p["spacing"])
        idx = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
        xyz_all = (idx - (m - 1) / 2.0) * a
        Z_all = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
        n_vac = int(round(p["vacancy_fraction"] * len(idx)))
        keep = np.sort(rng.permutation(len(idx))[n_vac:])
        xyz, Z = xyz_all[keep], Z_all[keep]
    elif kind == "neutral_ball":
        N = int(p["N"])
        xyz = _rsa(rng, N, _ball_attempts(p["radius"]), p["min_sep"])
        Z = np.concatenate([np.ones(N // 2), -np.ones(N - N // 2)])
        rng.shuffle(Z)
    else:
        raise ValueError(f"unknown particle kind {kind!r}")
    return Particles(np.ascontiguousarray(xyz, dtype=np.float64), np.ascontiguousarray(Z, dtype=np.float64))


@dataclass
class Request:
    arrival_s: float
    n: int
    particles: Particles


def make_serving_requests(cfg: dict, seed: int | None = None, count: int | None = None) -> list[Request]:
    """Poisson arrivals (exponential gaps), log-uniform particle counts, grid sizes
    drawn uniformly from a set; each request's particles follow ``uniform_box``."""
    s = cfg["serving"]
    rng = np.random.Generator(np.random.PCG64(seed_for(cfg["index"]) if seed is None else seed))
    cnt = int(s["requests"] if count is None else count)
    gaps = rng.exponential(s["mean_gap_ms"] * 1e-3, cnt)
    t = np.cumsum(gaps) - gaps[0]
    lo, hi = np.log(s["N_min"]), np.log(s["N_max"])
    Ns = np.floor(np.exp(rng.uniform(lo, hi, cnt))).astype(int)
    ns = rng.choice(np.asarray(s["n_choices"], int), size=cnt)
    seeds = rng.integers(0, 2**62, cnt)
    out = []
    for i in range(cnt):
        sub = {"particles": {"kind": "uniform_box", "N": int(Ns[i]), "half": s["half"],
                             "min_sep": s["min_sep"]}, "index": 0}
        out.append(Request(float(t[i]), int(ns[i]), make_particles(sub, seed=int(seeds[i]))))
    return out
