"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs.

Tolerances (relative Frobenius norms unless stated):
* same ranks, against the oracle's RS-Tucker tensor: both long-range parts lie within
  eps*||P_l|| of the untruncated P_l, and directions near the rank cut may mix differently in
  the two eigensolvers, so they agree within 2*eps*||P_l|| (relative to the grid) plus rounding:
  1e-9 for FP64, 1e-6 for FP32 (FP32 products, FP64-combined chunk sums in the core, FP32
  output);
* against the full-rank canonical sum P_0 of the oracle: eps * ||P_l|| / ||P_0|| (Tucker
  truncation) + the window cut-off (each window loses at most delta*|z| per point) + the
  rounding budget above;
* energy: 1e-8 (FP64) / 1e-6 (FP32) of sum_{j<k} |z_j z_k| / r_jk against the oracle's energy
  of the same RS tensor (Eq. (4.7)).
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


def _solve(cfg, xyz, Z, energy=True):
    ctx = _ctx(cfg, len(Z))
    ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"), energy=energy)
    torch.cuda.synchronize()
    return ctx


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def same_rank_tol(cfg, Pl, ref, rounding):
    """2*eps*||P_l|| / ||ref|| + rounding (see the module docstring)."""
    return 2 * cfg["eps"] * float(np.linalg.norm(Pl)) / float(np.linalg.norm(ref)) + rounding


@pytest.fixture(scope="module")
def c1():
    cfg = dict(load_config("c1_box64_n129"))
    cfg["rank_cap"] = 0
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    return cfg, p, pr


def test_c1_fp64_grid_matches_oracle_rs_tucker(c1):
    cfg, p, pr = c1
    ctx = _solve(cfg, p.xyz, p.Z)
    rep = ctx.report()
    P = ctx.potential.cpu().numpy()
    _, _, rk_or, _, _, _ = pr.tucker()
    assert all(abs(a - b) <= 1 for a, b in zip(rep["ranks"], rk_or)), (rep["ranks"], rk_or)
    assert rep["gamma"] == pr.gamma
    assert abs(rep["P_R0"] - pr.PR0) <= 1e-13 * pr.PR0
    Z0s, beta, _, _, _, _ = pr.tucker(ranks=rep["ranks"])
    ref = O.tucker_full(beta, Z0s) + pr.windows_grid()
    P0 = pr.P0_grid()
    Pl = pr.Pl_grid()
    assert _rel(P, ref) < same_rank_tol(cfg, Pl, ref, 1e-9)
    # against the untruncated canonical sum P_0
    bound = cfg["eps"] * np.linalg.norm(Pl) / np.linalg.norm(P0) + \
        pr.delta * np.sum(np.abs(pr.z)) * np.sqrt(P0.size) / np.linalg.norm(P0) + 1e-9
    assert _rel(P, P0) <= bound
    # energy of the same RS tensor (Eq. (4.7))
    E = ctx.energy()
    A = O.tucker_points(beta, Z0s, pr.j) + pr.windows_points(pr.j)
    Eref = O.energy_from_potential(A, pr.z, pr.PR0)
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    assert abs(E - Eref) <= 1e-8 * scale
    assert abs(E - pr.energy_P0()) <= 3 * cfg["eps"] * scale + 1e-6 * scale
    ctx.close()


def test_c1_rank_cap_reports_and_matches(c1):
    cfg, p, pr = c1
    cfg2 = dict(cfg)
    cfg2["rank_cap"] = 16
    ctx = _solve(cfg2, p.xyz, p.Z)
    rep = ctx.report()
    assert rep["status"] == 1 and rep["ranks"] == [16, 16, 16]
    Z0s, beta, _, _, _, _ = pr.tucker(ranks=[16, 16, 16])
    ref = O.tucker_full(beta, Z0s) + pr.windows_grid()
    # at the cap the retained energy is ~1e-4 of the tail, far from the mixing regime
    assert _rel(ctx.potential.cpu().numpy(), ref) < 1e-7
    ctx.close()


def test_tucker_factors_orthonormal_and_core(c1):
    cfg, p, pr = c1
    ctx = _solve(cfg, p.xyz, p.Z, energy=False)
    ranks, Vs, beta = ctx.tucker()
    for V in Vs:
        V = V.cpu().numpy()
        assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-12
    # projection identity: ||beta|| <= ||P_l|| and the gap is the Tucker error^2
    Pl = pr.Pl_grid()
    b = beta.cpu().numpy()
    gap = np.linalg.norm(Pl) ** 2 - np.sum(b * b)
    assert gap >= -1e-10 * np.linalg.norm(Pl) ** 2
    assert np.sqrt(max(gap, 0)) <= cfg["eps"] * np.linalg.norm(Pl)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_small_random_problems(prec):
    """Several tiles with ragged edges (n = 37, 45), windows that overlap and touch the
    boundary, mixed signs and a zero charge."""
    rng = np.random.default_rng(5)
    for n, N in ((37, 7), (45, 19)):
        cfg = dict(b=4.0, n=n, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0,
                   delta_rel=1e-8, precision=prec, snap=True)
        xyz = rng.uniform(-4.0, 4.0, (N, 3))
        xyz[0] = [-4.0, 4.0, 0.0]
        Z = rng.uniform(-1, 1, N)
        Z[1] = 0.0
        pr = O.Problem(cfg, xyz, Z)
        ctx = _solve(cfg, xyz, Z)
        rep = ctx.report()
        Z0s, beta, _, _, _, _ = pr.tucker(ranks=rep["ranks"])
        ref = O.tucker_full(beta, Z0s) + pr.windows_grid()
        tol = same_rank_tol(cfg, pr.Pl_grid(), ref, 1e-9 if prec == "fp64" else 1e-6)
        assert _rel(ctx.potential.double().cpu().numpy(), ref) < tol, (n, N)
        P0 = pr.P0_grid()
        bound = cfg["eps"] * np.linalg.norm(pr.Pl_grid()) / np.linalg.norm(P0) + \
            pr.delta * np.sum(np.abs(pr.z)) * np.sqrt(P0.size) / np.linalg.norm(P0) + \
            (1e-9 if prec == "fp64" else 1e-6)
        assert _rel(ctx.potential.double().cpu().numpy(), P0) <= bound, (n, N)
        A = O.tucker_points(beta, Z0s, pr.j) + pr.windows_points(pr.j)
        Eref = O.energy_from_potential(A, pr.z, pr.PR0)
        assert abs(ctx.energy() - Eref) <= (1e-8 if prec == "fp64" else 1e-6) * O.energy_scale(pr.xyz_snapped, pr.z)
        ctx.close()


def test_eval_points_matches_grid(c1):
    cfg, p, pr = c1
    ctx = _solve(cfg, p.xyz, p.Z, energy=False)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, pr.n, (500, 3))
    v = ctx.eval_points(torch.tensor(idx, dtype=torch.int32)).cpu().numpy()
    P = ctx.potential.cpu().numpy()
    g = P[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.max(np.abs(v - g)) <= 1e-10 * np.max(np.abs(P))
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_edge_cases_empty_zero_and_single(prec):
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision=prec, snap=True)
    rnd = 1e-9 if prec == "fp64" else 1e-6
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    ctx = RSContext(config_from_workload(cfg, max_particles=4))
    # empty input
    ctx.solve(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
              torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert float(ctx.potential.abs().max()) == 0.0 and ctx.energy() == 0.0
    # all charges zero
    ctx.solve(torch.tensor([[0.5, 0.5, 0.5]], dtype=torch.float64, device="cuda"),
              torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert float(ctx.potential.abs().max()) == 0.0 and ctx.energy() == 0.0
    # a single charge: no interaction energy; potential equals the oracle
    xyz = np.array([[1.0, -2.0, 0.25]])
    Z = np.array([0.8])
    ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"))
    pr = O.Problem(cfg, xyz, Z)
    rep = ctx.report()
    Z0s, beta, _, _, _, _ = pr.tucker(ranks=rep["ranks"])
    ref = O.tucker_full(beta, Z0s) + pr.windows_grid()
    Pg = ctx.potential.double().cpu().numpy()
    assert _rel(Pg, ref) < same_rank_tol(cfg, pr.Pl_grid(), ref, rnd)
    Eref = O.energy_from_potential(O.tucker_points(beta, Z0s, pr.j) + pr.windows_points(pr.j), pr.z, pr.PR0)
    assert abs(ctx.energy() - Eref) <= rnd * pr.PR0 * Z[0] ** 2
    # the host input path gives the same result bit for bit (every floating-point sum of a
    # solve has a fixed order)
    P1 = ctx.potential.clone()
    E1 = ctx.energy()
    ctx.solve(xyz, Z)
    torch.cuda.synchronize()
    assert torch.equal(P1, ctx.potential)
    assert ctx.energy() == E1
    ctx.close()


def test_invalid_inputs_raise():
    from paper_1606_09218_gb300 import RSContext, RSError, config_from_workload
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp64", snap=True)
    ctx = RSContext(config_from_workload(cfg, max_particles=2))
    with pytest.raises(RSError):
        ctx.solve(np.array([[5.0, 0.0, 0.0]]), np.array([1.0]))          # outside the box
    with pytest.raises(RSError):
        ctx.solve(np.zeros((3, 3)), np.ones(3))                           # above capacity
    # device-side detection of an outside centre
    ctx.solve(torch.tensor([[0.0, 0.0, 9.0]], dtype=torch.float64, device="cuda"),
              torch.ones(1, dtype=torch.float64, device="cuda"))
    with pytest.raises(RSError):
        ctx.energy()
    # separation check
    ctx.solve(np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0]]), np.array([1.0, -1.0]), min_sep=0.5)
    with pytest.raises(RSError):
        ctx.report()
    ctx.close()
    bad = config_from_workload(dict(cfg, n=32), max_particles=2)
    with pytest.raises(RSError):
        RSContext(bad)


def test_c2_full_size_sampled_against_canonical_sum():
    """Config 2 at full size (n = 513, N = 1000, FP32 bulk, eps = 1e-6: the configuration the
    throughput is quoted on), in the launch configuration the benchmark times: the grid against
    the oracle's full-rank canonical sum P_0 (no split, no truncation) at every particle site and
    4000 random grid points.  The relative error over the sample is bounded by the split
      eps ||P_l|| / ||P_0||            (Tucker truncation of the long part, Sec. 6)
    + delta sum|z| sqrt(M) / ||P_0||   (window cut-off, Sec. 2.3 criterion (A))
    + 1e-6                             (FP32 bulk arithmetic)
    with the norms taken over the sample, and it stays within the stated 1e-6 itself.  The energy
    (Eq. (4.7)) is compared with the energy of P_0 at the stated tolerance of the energy scale."""
    cfg = load_config("c2_protein1000_n513")
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _solve(cfg, p.xyz, p.Z)
    rep = ctx.report()
    assert rep["status"] == 0
    P = ctx.potential
    rng = np.random.default_rng(17)
    idx = np.concatenate([pr.j, rng.integers(0, pr.n, (4000, 3))])
    it = torch.tensor(idx, device="cuda", dtype=torch.long)
    g = P[it[:, 0], it[:, 1], it[:, 2]].double().cpu().numpy()
    ref = pr.P0_points(idx)
    Pl = pr.Pl_points(idx)
    nref = float(np.linalg.norm(ref))
    tucker = cfg["eps"] * float(np.linalg.norm(Pl)) / nref
    window = pr.delta * float(np.sum(np.abs(pr.z))) * np.sqrt(len(idx)) / nref
    err = _rel(g, ref)
    print(f"c2 full size: sample error {err:.3e} (Tucker {tucker:.2e}, window {window:.2e}, rounding 1e-6)")
    assert err <= tucker + window + 1e-6, err
    assert err < 1e-6, err
    E = ctx.energy()
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    dE = abs(E - pr.energy_P0()) / scale
    print(f"c2 full size: energy error {dE:.3e} of the energy scale")
    assert dE <= 1e-6, dE
    ctx.close()


def test_c3_full_size_sampled_against_canonical_sum():
    """Config 3 at full size (n = 1025, N = 19,757 lattice sites, eps = 1e-5, FP32 bulk; the
    large Tucker rank leaves room for one T2 stage and four window slots, with the epilogue
    storing from registers): the grid against the oracle's full-rank canonical sum on sampled
    sites and points, and the energy against the grid at all sites (E = 1/2 sum_j z_j (P(x_j) -
    z_j P_R(0)), Eq. (4.7), a property that holds at any size)."""
    cfg = load_config("c3_nacl28_n1025")
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _solve(cfg, p.xyz, p.Z)
    rep = ctx.report()
    assert rep["status"] == 0
    assert max(rep["tail_rel"]) <= cfg["eps"] ** 2 / 3 * 1.0001
    P = ctx.potential
    rng = np.random.default_rng(23)
    idx = np.concatenate([pr.j[rng.choice(len(p.Z), 300, replace=False)], rng.integers(0, pr.n, (300, 3))])
    it = torch.tensor(idx, device="cuda", dtype=torch.long)
    g = P[it[:, 0], it[:, 1], it[:, 2]].double().cpu().numpy()
    ref = pr.P0_points(idx)
    err = _rel(g, ref)
    assert err < cfg["eps"], err
    js = torch.tensor(pr.j, device="cuda", dtype=torch.long)
    at_sites = P[js[:, 0], js[:, 1], js[:, 2]].double().cpu().numpy()
    E_grid = 0.5 * float(np.sum(pr.z * (at_sites - pr.z * rep["P_R0"])))
    scale = float(np.abs(pr.z).sum() * np.abs(at_sites).max())
    assert abs(ctx.energy() - E_grid) <= 1e-6 * scale
    ctx.close()


@pytest.mark.parametrize("name", ["c2_protein1000_n513"])
def test_tensor_core_reconstruction_matches_cuda_core_path(name, monkeypatch):
    """The tcgen05 (3xTF32) assembly (Tucker product and windows in one kernel) against the
    FP32 CUDA-core product followed by the window kernel, on the same input: both approximate
    the same FP32 sums; the split products keep the difference at the 1e-7 level (well inside the
    1e-6 parity budget).  The path is chosen when a context is created."""
    cfg = load_config(name)
    p = make_particles(cfg)
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    monkeypatch.setenv("RS_RECON_PATH", "cuda")
    cref = _ctx(cfg, len(p.Z))
    cref.solve(xyz, Z, energy=False)
    ref = cref.potential.clone()
    rref = cref.report()
    cref.close()
    monkeypatch.setenv("RS_RECON_PATH", "tc")
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(xyz, Z, energy=False)
    torch.cuda.synchronize()
    rep = ctx.report()
    assert rep["status"] == 0
    assert rep["ranks"] == rref["ranks"] and rep["gamma"] == rref["gamma"]
    # the assembly replaces the product and window kernels by one kernel plus the list builders
    assert rep["kernel_launches"] != rref["kernel_launches"]
    P = ctx.potential
    d = float((P.double() - ref.double()).norm() / ref.double().norm())
    assert d < 1e-6, d
    # spot values at the grid corners and the last (ragged) row and column
    n = ref.shape[0]
    for i in ((0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n - 1), (127, 255, 256), (128, 300, 5)):
        a, b = float(P[i]), float(ref[i])
        assert abs(a - b) <= 1e-5 * max(1.0, abs(b)), (i, a, b)
    ctx.close()


@pytest.mark.parametrize("path", ["kr", "tc"])
def test_tensor_core_core_matches_cuda_core_path(monkeypatch, path):
    """The two tcgen05 forms of the core contraction (FP16-split operands, 64-term FP32 segments
    folded into two-sums, fixed-point sums across work units) forced on config 2 against the
    CUDA-core FP32 contraction with two-sum chunks: the same Tucker ranks, and potentials within
    1e-6 (the tensor cores' FP32 accumulation costs about 4e-7 here).  "kr" forms the Khatri-Rao
    operand z q1 q2 once per solve and streams it (the default on the FP32 path); "tc" builds
    both operands per output tile."""
    cfg = load_config("c2_protein1000_n513")
    p = make_particles(cfg)
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    monkeypatch.setenv("RS_CORE_PATH", "cuda")
    cref = _ctx(cfg, len(p.Z))
    cref.solve(xyz, Z, energy=True)
    ref = cref.potential.clone()
    Eref = cref.energy()
    rref = cref.report()
    cref.close()
    monkeypatch.setenv("RS_CORE_PATH", path)
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(xyz, Z, energy=True)
    rep = ctx.report()
    assert rep["status"] == 0 and rep["ranks"] == rref["ranks"]
    if path == "tc":
        assert rep["kernel_launches"] == rref["kernel_launches"] + 1       # + the K-term table
    else:
        # + the K-term table, and per window of K an operand kernel and an MMA kernel
        extra = rep["kernel_launches"] - rref["kernel_launches"]
        assert extra >= 2 and extra % 2 == 0, extra
    d = float((ctx.potential.double() - ref.double()).norm() / ref.double().norm())
    assert d < 1e-6, d
    pr = O.Problem(cfg, p.xyz, p.Z)
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    assert abs(ctx.energy() - Eref) <= 3e-7 * scale
    ctx.close()


def test_khatri_rao_core_over_windows_and_c_tiles(monkeypatch):
    """The forces workload (N = 4096, r = 66, snapped): its Khatri-Rao operands take several
    windows of K, and r3 > 64 puts c in one tile of 96 values.  Against the CUDA-core contraction: the same
    ranks, potentials within 1e-6, the energy within 3e-7 of its scale, and a repeated solve
    bit-identical (fixed-point sums)."""
    cfg = dict(load_config("c5_forces4096_n513"), snap=True)
    p = make_particles(cfg)
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    monkeypatch.setenv("RS_CORE_PATH", "cuda")
    cref = _ctx(cfg, len(p.Z))
    cref.solve(xyz, Z, energy=True)
    ref = cref.potential.clone()
    Eref = cref.energy()
    rref = cref.report()
    cref.close()
    monkeypatch.setenv("RS_CORE_PATH", "kr")
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(xyz, Z, energy=True)
    rep = ctx.report()
    assert rep["status"] == 0 and rep["ranks"] == rref["ranks"] and max(rep["ranks"]) > 64
    assert rep["kernel_launches"] - rref["kernel_launches"] >= 4          # two windows at least
    P1 = ctx.potential.clone()
    d = float((P1.double() - ref.double()).norm() / ref.double().norm())
    assert d < 1e-6, d
    pr = O.Problem(cfg, p.xyz, p.Z)
    assert abs(ctx.energy() - Eref) <= 3e-7 * O.energy_scale(pr.xyz_snapped, pr.z)
    ctx.solve(xyz, Z, energy=True)
    assert torch.equal(ctx.potential, P1)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_plain_method_paths_match_oracle(prec):
    """The plain-method GPU paths on the last solve's particles: the direct sum Z / r against
    the oracle's direct analytic sum (terms at r = 0 skipped) and the full-rank canonical sum
    against the oracle's P_0, both on the whole grid (FP32 products, compensated sums)."""
    rng = np.random.default_rng(31)
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision=prec, snap=True)
    N = 12
    xyz = rng.uniform(-3.0, 3.0, (N, 3))
    Z = rng.uniform(-1, 1, N)
    Z[5] = 0.0
    pr = O.Problem(cfg, xyz, Z)
    ctx = _solve(cfg, xyz, Z)
    D = ctx.plain_direct().double().cpu().numpy().ravel()
    C0 = ctx.plain_canonical().double().cpu().numpy().ravel()
    n = cfg["n"]
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    Dref = O.direct_sum_points(pr.xyz_snapped, pr.z, pr.x[idx])
    Cref = pr.P0_grid().ravel()
    assert _rel(D, Dref) < 1e-6
    assert np.abs(D - Dref).max() <= 2e-6 * np.abs(Dref).max()
    assert _rel(C0, Cref) < 1e-6
    assert np.abs(C0 - Cref).max() <= 2e-6 * np.abs(Cref).max()
    ctx.close()


# ---------------------------------------------------------------- forces (Sec. 4.3)
def _forces_tol(cfg, rounding):
    """Both the GPU and the oracle RS-Tucker forces are within O(eps) of the untruncated forces
    (oracle pins: about 6 eps for the discrete gradient, 1e-5 at eps = 1e-6 for the adjoint of
    the continued basis); 20*eps covers both, plus the rounding of the bulk precision."""
    return 20 * cfg["eps"] + rounding


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_forces_discrete_gradient_match_oracle(prec):
    """Forces through the C ABI from the discrete gradient of the RS-Tucker tensor (Sec. 4.3,
    Eq. (4.9)): against the oracle's discrete gradient of its own RS-Tucker tensor at the same
    ranks and of the untruncated long-range sum (both within O(eps) of each other, element by
    element in the norm of the forces), against the analytic derivative of the untruncated kernel
    within the same bound (the order-8 difference formula adds far less); zero-charge particles
    get zero force, the total force is nearly zero, and a particle on the boundary of the box
    (one-sided rows) is covered."""
    rng = np.random.default_rng(12)
    cfg = dict(b=4.0, n=45, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision=prec, snap=True)
    N = 16
    xyz = rng.uniform(-3.2, 3.2, (N, 3))
    xyz[5] = [-4.0, 0.3, 3.9]
    Z = rng.uniform(-1, 1, N)
    Z[3] = 0.0
    pr = O.Problem(cfg, xyz, Z)
    ctx = _ctx(cfg, N)
    ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"), forces=True)
    F = ctx.forces().cpu().numpy()
    rep = ctx.report()
    assert rep["status"] == 0
    Ft, _ = pr.forces_rs_tucker_fd(ranks=rep["ranks"])
    Fc = pr.forces_canonical_fd()
    Fa = pr.forces_direct_long()
    rounding = 1e-10 if prec == "fp64" else 2e-6
    tol = _forces_tol(cfg, rounding)
    scale = np.abs(Fc).max()
    assert np.abs(F - Ft).max() <= tol * scale
    assert np.abs(F - Fc).max() <= tol * scale
    assert np.linalg.norm(F - Fa) / np.linalg.norm(Fa) < tol
    assert np.all(F[3] == 0.0)
    assert np.abs(F.sum(0)).max() <= tol * scale * N
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_forces_pair_kernel_match_oracle(prec):
    """RS_FORCES_PAIR: the untruncated long-range pair kernel plus the windows, against the
    oracle's direct form element by element (FP64 products: 1e-10; FP32 products: 2e-6), and
    against the oracle's RS-Tucker forces at the same ranks and the forces of the untruncated
    Galerkin kernel (both within O(eps))."""
    rng = np.random.default_rng(12)
    cfg = dict(b=4.0, n=45, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision=prec, snap=True)
    N = 16
    xyz = rng.uniform(-3.2, 3.2, (N, 3))
    Z = rng.uniform(-1, 1, N)
    Z[3] = 0.0
    pr = O.Problem(cfg, xyz, Z)
    ctx = _ctx(cfg, N)
    ctx.solve(torch.tensor(xyz, device="cuda"), torch.tensor(Z, device="cuda"), forces=True, forces_pair=True)
    F = ctx.forces().cpu().numpy()
    rep = ctx.report()
    assert rep["status"] == 0
    Fd = pr.forces_direct_long()
    Fo = pr.forces_rs_tucker(ranks=rep["ranks"])[0]
    Fg = pr.forces_galerkin()
    rounding = 1e-10 if prec == "fp64" else 2e-6
    assert np.abs(F - Fd).max() <= rounding * np.abs(Fd).max()
    tol = _forces_tol(cfg, rounding)
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < tol
    assert np.linalg.norm(F - Fg) / np.linalg.norm(Fg) < tol
    assert np.all(F[3] == 0.0)
    assert np.abs(F.sum(0)).max() <= tol * np.abs(F).max() * N
    ctx.close()


@pytest.mark.parametrize("name", ["c2_protein1000_n513", "c5_forces4096_n513"])
def test_forces_full_size_sampled(name):
    """Full size, FP32 bulk (the protein workload, and the forces workload's N = 4096 at snapped
    centres): the discrete-gradient forces against the oracle's discrete gradient of the
    untruncated long-range sum (plus windows) on a sample of particles, and against the forces of
    the untruncated Galerkin kernel; O(eps) bounds as above."""
    cfg = dict(load_config(name), snap=True)
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"), forces=True,
              want_potential=False)
    F = ctx.forces().cpu().numpy()
    assert ctx.report()["status"] == 0
    sel = np.nonzero(pr.z != 0)[0][::29]
    D = pr.fd_matrix()
    G = O.canonical_fd_gradient_points(pr.j, pr.z, pr.pk, pr.klong, D, pr.j[sel])
    G -= pr.z[sel, None] * O.fd_self_gradient(pr.j[sel], pr.pk, pr.klong, D)
    dpk = O.reference_factor_derivatives(pr.t, pr.a, pr.h, pr.n)
    Fw = O._window_forces(pr.j, pr.z, pr.pk, dpk, pr.kshort, pr.gamma, pr.n)[sel]
    Fc = -pr.z[sel, None] * G + Fw
    tol = _forces_tol(cfg, 2e-6)
    err = np.linalg.norm(F[sel] - Fc) / np.linalg.norm(Fc)
    print(f"{name}: discrete-gradient forces vs the oracle's untruncated discrete gradient {err:.2e}")
    assert err < tol, err
    Fg = pr.forces_galerkin()
    err_g = np.linalg.norm(F[sel] - Fg[sel]) / np.linalg.norm(Fg[sel])
    assert err_g < tol, err_g
    ctx.close()


def test_forces_autograd_and_not_ready():
    """rs_energy(...).backward() puts -F into xyz.grad; asking for forces of a solve that did
    not compute them is an error."""
    from paper_1606_09218_gb300 import RSError, rs_energy
    rng = np.random.default_rng(8)
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp64", snap=True)
    xyz = torch.tensor(rng.uniform(-2.5, 2.5, (5, 3)), device="cuda", requires_grad=True)
    Z = torch.tensor(rng.uniform(-1, 1, 5), device="cuda")
    ctx = _ctx(cfg, 5)
    E = rs_energy(xyz, Z, ctx)
    E.backward()
    F = ctx.forces()
    assert torch.allclose(xyz.grad, -F)
    assert abs(float(E.detach()) - ctx.energy()) == 0.0
    ctx.solve(xyz.detach(), Z, forces=False)
    with pytest.raises(RSError):
        ctx.forces()
    ctx.close()


# ---------------------------------------------------------------- short-range part (rs_get_windows)
def _windows_from_table(gamma, f, j, z, n):
    """W[i] = sum_nu z_nu sum_k f_k[i1 - j1 + g] f_k[i2 - j2 + g] f_k[i3 - j3 + g] over the
    centres whose window reaches i (Def. 3.6), assembled on the host from the returned table."""
    W = np.zeros((n, n, n))
    g = gamma
    for q in range(len(z)):
        if z[q] == 0.0:
            continue
        lo = [max(0, j[q, l] - g) for l in range(3)]
        hi = [min(n - 1, j[q, l] + g) for l in range(3)]
        sl = [f[:, lo[l] - j[q, l] + g: hi[l] - j[q, l] + g + 1] for l in range(3)]
        W[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] += z[q] * np.einsum("ka,kb,kc->abc", *sl)
    return W


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_get_windows_rebuilds_oracle_short_range_part(c1, prec):
    """rs_get_windows returns the uniform cumulated canonical tensor of the short-range part
    (Defs. 3.4, 3.6): its factor table equals the oracle's short-range factors on -gamma..gamma,
    the centres are the oracle's snapped indices, and the part rebuilt from the table on the host
    equals the oracle's windows on the whole grid, element by element."""
    cfg, p, pr = c1
    cfg = dict(cfg, precision=prec)
    ctx = _solve(cfg, p.xyz, p.Z, energy=False)
    gamma, f, j, z = ctx.windows()
    assert gamma == pr.gamma and f.shape == (cfg["R_s"], 2 * gamma + 1)
    n = pr.n
    fo = pr.pk[pr.kshort][:, n - 1 - gamma: n + gamma]
    f = f.cpu().numpy()
    assert np.abs(f - fo).max() <= 1e-14 * np.abs(fo).max()
    j = j.cpu().numpy()
    assert np.array_equal(j, pr.j)
    assert np.array_equal(z.cpu().numpy(), p.Z)
    W = _windows_from_table(gamma, f, j, p.Z, n)
    Wo = pr.windows_grid()
    assert np.abs(W - Wo).max() <= 1e-13 * np.abs(Wo).max()
    ctx.close()


def test_get_windows_needs_a_solve_and_follows_the_last_one():
    from paper_1606_09218_gb300 import RSContext, RSError, config_from_workload
    cfg = dict(b=4.0, n=33, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp32_split", snap=True)
    ctx = RSContext(config_from_workload(cfg, max_particles=3))
    with pytest.raises(RSError):
        ctx.windows()
    xyz = np.array([[0.5, -1.0, 2.0], [-2.0, 1.5, 0.0]])
    ctx.solve(xyz, np.array([0.7, -0.3]), energy=False)
    g, f, j, z = ctx.windows()
    assert j.shape == (2, 3) and z.shape == (2,) and f.shape[0] == 4
    ctx.solve(xyz[:1], np.array([0.2]), energy=False)
    g2, f2, j2, z2 = ctx.windows()
    assert j2.shape == (1, 3) and float(z2[0]) == 0.2 and g2 == g
    ctx.close()
