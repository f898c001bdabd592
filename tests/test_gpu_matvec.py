"""GPU tests of the RS interaction matrix (rs_matvec, rs_energy_matvec; Sec. 4.1 problem (B)
case (A), Sec. 4.2 Eq. (4.6)) against the oracle's dense matrix and its RS tensor.

Tolerances: the FP64 context computes the FFTs in FP64 (rounding ~1e-15 of the result's
largest entry per mode product, 3R products: 1e-12 here); the FP32 context in FP32 (~1e-7 per
product: 5e-6 of the largest entry).  The energy: 1e-10 (FP64) and 1e-6 (FP32) of the energy
scale sum |z_j z_k| / r_jk.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_split": 5e-6}
ETOL = {"fp64": 1e-10, "fp32_split": 1e-6}


def _ctx(cfg, N):
    from paper_1606_09218_gb300 import RSContext, config_from_workload
    return RSContext(config_from_workload(cfg, max_particles=max(1, N)))


def _small(prec, n):
    return dict(b=2.0, n=n, R=10, R_s=3, h_q=0.8, u0=-4.0, eps=1e-6, rank_cap=0, delta_rel=1e-6,
                precision=prec, snap=True)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
@pytest.mark.parametrize("n", [11, 17])
def test_matvec_matches_the_dense_matrix(prec, n):
    """Y = A X for a random X on two grids (n = 11: a circulant of 32 > 2n - 2 points; n = 17: of
    exactly 2n - 2 = 32 points, where the offsets +-(n-1) share one entry), every selection of
    terms, with and without the diagonal."""
    cfg = _small(prec, n)
    pr = O.Problem(cfg, np.zeros((1, 3)), np.zeros(1))
    ctx = _ctx(cfg, 1)
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n, n))
    Xd = torch.tensor(X, device="cuda", dtype=ctx.dtype)
    Xr = Xd.double().cpu().numpy()
    for long, short, sel in ((True, True, (pr.klong, pr.kshort)), (True, False, (pr.klong, [])),
                             (False, True, ([], pr.kshort))):
        for off in (False, True):
            Y = ctx.matvec(Xd, long=long, short=short, offdiag=off).double().cpu().numpy()
            ref = O.rs_matvec_dense(pr.pk, np.asarray(sel[0], int), np.asarray(sel[1], int), pr.gamma, n, Xr,
                                    offdiag=off)
            err = np.abs(Y - ref).max() / np.abs(ref).max()
            assert err <= TOL[prec], (long, short, off, err)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_matvec_of_the_charges_is_the_rs_tensor(prec):
    """A applied to the charges embedded in a 45^3 grid (M = 128, several CTAs per mode, ragged
    fibre batches) equals the oracle's untruncated long-range canonical sum plus its windows,
    element by element."""
    rng = np.random.default_rng(19)
    cfg = dict(b=4.0, n=45, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision=prec, snap=True)
    N = 19
    xyz = rng.uniform(-4.0, 4.0, (N, 3))
    xyz[0] = [-4.0, 4.0, 0.0]
    Z = rng.uniform(-1, 1, N)
    pr = O.Problem(cfg, xyz, Z)
    ctx = _ctx(cfg, N)
    C = torch.tensor(O.charge_grid(pr.j, pr.z, pr.n), device="cuda", dtype=ctx.dtype)
    Y = ctx.matvec(C).double().cpu().numpy()
    ref = pr.Pl_grid() + pr.windows_grid()
    assert np.abs(Y - ref).max() <= TOL[prec] * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("name,prec", [("c1_box64_n129", "fp64"), ("c2_protein1000_n513", "fp32_split")])
def test_energy_through_the_matrix_matches_oracle(name, prec):
    """E_N = 1/2 <(A - diag A) z, z> (Eq. (4.6)) of the last solve's charges against the oracle's
    energy of the same untruncated RS tensor (Eq. (4.7) with the canonical long-range sum and the
    windows at the particles), and within the Tucker tolerance of the solve's RS-Tucker energy."""
    cfg = dict(load_config(name), precision=prec, rank_cap=0)
    p = make_particles(cfg)
    pr = O.Problem(cfg, p.xyz, p.Z)
    ctx = _ctx(cfg, len(p.Z))
    ctx.solve(torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"), energy=True,
              want_potential=False)
    E_rs = ctx.energy()
    E = ctx.energy_matvec()
    ref = O.energy_from_potential(pr.Pl_points(pr.j) + pr.windows_points(pr.j), pr.z, pr.PR0)
    scale = O.energy_scale(pr.xyz_snapped, pr.z)
    print(f"{name}: energy through the matrix {E:.12f}, oracle {ref:.12f}, RS-Tucker {E_rs:.12f}")
    assert abs(E - ref) <= ETOL[prec] * scale
    assert abs(E - E_rs) <= 3 * cfg["eps"] * scale + ETOL[prec] * scale
    # a second call gives the same value (the scratch grids are cleared)
    assert ctx.energy_matvec() == E
    ctx.close()


def test_matvec_arguments_and_readiness():
    from paper_1606_09218_gb300 import RSError
    cfg = _small("fp64", 11)
    ctx = _ctx(cfg, 1)
    X = torch.zeros((11, 11, 11), dtype=torch.float64, device="cuda")
    with pytest.raises(RSError):
        ctx.energy_matvec()                    # no solve yet
    with pytest.raises(RSError):
        ctx.matvec(X, Y=X)                     # in place is not allowed
    assert float(ctx.matvec(X).abs().max()) == 0.0
    ctx.close()


@pytest.mark.parametrize("n", [33, 129, 257, 601])
def test_matvec_fp32_transform_sizes(n):
    """The FP32 transform for the circulant sizes 32 P with P = 2, 8, 16, 64 (n = 601 takes the
    2048-point circulant): A applied to the charges equals the oracle's long-range canonical sum
    plus the windows, on the whole grid (n = 33) or at the particle sites and 2000 random grid
    points."""
    rng = np.random.default_rng(n)
    b = 4.0 * (n - 1) / 32
    cfg = dict(b=b, n=n, R=14, R_s=4, h_q=0.7, u0=-6.5, eps=1e-6, rank_cap=0, delta_rel=1e-8,
               precision="fp32_split", snap=True)
    N = 24
    xyz = rng.uniform(-0.9 * b, 0.9 * b, (N, 3))
    Z = rng.uniform(-1, 1, N)
    pr = O.Problem(cfg, xyz, Z)
    ctx = _ctx(cfg, N)
    C = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    jt = torch.tensor(pr.j, device="cuda", dtype=torch.long)
    C.index_put_((jt[:, 0], jt[:, 1], jt[:, 2]), torch.tensor(pr.z, device="cuda", dtype=torch.float32),
                 accumulate=True)
    Y = ctx.matvec(C)
    if n <= 33:
        ref = pr.Pl_grid() + pr.windows_grid()
        got = Y.double().cpu().numpy()
    else:
        idx = np.concatenate([pr.j, rng.integers(0, n, (2000, 3))])
        it = torch.tensor(idx, device="cuda", dtype=torch.long)
        got = Y[it[:, 0], it[:, 1], it[:, 2]].double().cpu().numpy()
        ref = pr.Pl_points(idx) + pr.windows_points(idx)
    assert np.abs(got - ref).max() <= TOL["fp32_split"] * np.abs(ref).max(), n
    ctx.close()
